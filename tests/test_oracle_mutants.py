"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of oracle/oracle.cpp with one planted mistake (a
dropped term, a wrong sign, index or operand, a wrong schedule) and checks
that at least one pin fails on it. Mistakes are planted on the CPU only.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, jmask_bool, neighbours
from tests.test_oracle_sweep_sets import face_sets_hold, reflected_blocks_hold
from tests.test_oracle_tables6to8 import decomposed_within_table6
from tests.test_oracle_procedure import procedure3d_holds, procedure_holds

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")


def _build_mutant(tmp_path, anchor, replacement):
    src = open(SRC).read()
    assert src.count(anchor) == 1, f"anchor not unique/found: {anchor!r}"
    path = tmp_path / "mut.cpp"
    path.write_text(src.replace(anchor, replacement))
    out = str(tmp_path / "libmut.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", out,
                    str(path)], check=True)
    return oracle.lib(out)


def _rand_diags(n, stencil, seed):
    g = np.random.default_rng(seed)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(stencil, N))
    d[neighbours(full_n(n), stencil) < 0] = 0.0
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, size=N)
    return d


# --- detectors: return True when the pin holds --------------------------------

def pin_table1_pgs2(L):
    n = 39
    d, b = W.laplace1d(n)
    pb = oracle.Problem(1, (n,), 3, d, (2,), library=L)
    x, exact, k = np.zeros(n), np.arange(1, n + 1) / 40, 0
    while k < 3000:
        x = pb.sor_sweep(oracle.DECOMPOSED, k, 1.0, b, x)
        k += 1
        if np.abs(x - exact).sum() / 41 < 1e-3:
            break
    return k == 975


def pin_splitting(L):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n, stencil, sub = (13, 11, 1), 5, (2, 2)
    d = _rand_diags(n, stencil, 3)
    N = 143
    g = np.random.default_rng(1)
    pb = oracle.Problem(2, n, stencil, d, sub, library=L)
    omega = np.array([0.7, 1.3, 1.6, 0.9])
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    for t in range(4):
        x = pb.sor_sweep(oracle.DECOMPOSED, t, omega, b, u)
        jm, corner, _, _ = pb.plan_info(oracle.DECOMPOSED, t)
        J = jmask_bool(jm, stencil)
        U = ~J & (neighbours(n, stencil) >= 0)
        U[0] = False
        w = omega[corner]
        lhs = (sp.diags(d[0]) + sp.diags(w) @ assemble(n, stencil, d, J, False)).tocsc()
        rhs = (sp.diags((1 - w) * d[0]) - sp.diags(w) @ assemble(n, stencil, d, U, False)) @ u + w * b
        if not np.allclose(x, spla.spsolve(lhs, rhs), rtol=0, atol=1e-12):
            return False
    return True


def pin_printed_systems(L):
    n = (6, 6, 1)
    pb = oracle.Problem(2, n, 5, W.poisson2d(6, 6), (2, 2), library=L)
    jm, corner, nblocks, mb = pb.plan_info(oracle.DECOMPOSED, 0)
    J = lambda x, y: {k for k in range(1, 5) if int(jm[x + 6 * y]) >> k & 1}
    return (J(2, 2) == {2, 4} and J(3, 2) == {1, 4} and J(1, 2) == {2, 4} and mb == 4
            and int(corner[7]) == 3 and int(corner[10]) == 2)


def pin_schedule(L):
    return [L.orc_base_corner(2, t) for t in range(4)] == [3, 0, 2, 1]


def pin_ssor_symmetric(L):
    n = (11, 9, 1)
    d = _rand_diags(n, 5, 61)
    pb = oracle.Problem(2, n, 5, d, (2, 3), library=L)
    g = np.random.default_rng(2)
    r1, r2 = g.uniform(-1, 1, 99), g.uniform(-1, 1, 99)
    z1, z2 = pb.ssor_apply(oracle.DECOMPOSED, 1.3, r1), pb.ssor_apply(oracle.DECOMPOSED, 1.3, r2)
    return abs(z1 @ r2 - z2 @ r1) <= 1e-13 * np.linalg.norm(z1) * np.linalg.norm(r2)


def pin_ilu_pattern(L, mode):
    n, stencil = (9, 7, 1), 5
    d = _rand_diags(n, stencil, 31)
    pb = oracle.Problem(2, n, stencil, d, (1, 1) if mode == 0 else (3, 2), library=L)
    try:
        pb.ilu0_factor(mode)
    except RuntimeError:
        return False
    A = assemble(n, stencil, d).toarray()
    nb = neighbours(n, stencil)
    if mode == 0:
        f = pb.ilu0_export()
        idx = np.arange(63)
        Lm = assemble(n, stencil, f, (nb >= 0) & (nb < idx), False).toarray() + np.eye(63)
        Um = assemble(n, stencil, f, nb > idx, True).toarray()
        M = Lm @ Um
    else:
        dt = pb.ilu0_export()
        tf = pb.fwd_phase()
        Jf = jmask_bool(pb.plan_info(1, tf)[0], stencil)
        Jb = jmask_bool(pb.plan_info(1, tf ^ 1)[0], stencil)
        M = (np.diag(dt) + assemble(n, stencil, d, Jf, False).toarray()) @ np.diag(1 / dt) @ \
            (np.diag(dt) + assemble(n, stencil, d, Jb, False).toarray())
    return np.max(np.abs((M - A)[A != 0])) <= 1e-12


def pin_dilu9(L):
    """9-point decomposed D-ILU: M = (D~ + L) D~^-1 (D~ + U) has A's diagonal."""
    n = (13, 11, 1)
    d = _rand_diags(n, 9, 51)
    pb = oracle.Problem(2, n, 9, d, (3, 2), library=L)
    try:
        pb.ilu0_factor(oracle.DECOMPOSED)
    except RuntimeError:
        return False
    dt = pb.ilu0_export()
    tf = pb.fwd_phase()
    Jf = jmask_bool(pb.plan_info(1, tf)[0], 9)
    Jb = jmask_bool(pb.plan_info(1, tf ^ 1)[0], 9)
    M = (np.diag(dt) + assemble(n, 9, d, Jf, False).toarray()) @ np.diag(1 / dt) @ \
        (np.diag(dt) + assemble(n, 9, d, Jb, False).toarray())
    A = assemble(n, 9, d).toarray()
    return np.max(np.abs(np.diag(M) - np.diag(A))) <= 1e-14 * np.max(np.abs(np.diag(A)))

def pin_krylov_counts(L, method):
    from tests.test_oracle_pins import krylov_counts_match_scipy
    try:
        return krylov_counts_match_scipy(L, method)
    except RuntimeError:
        return False


def pin_table5_ssour(L):
    # Table 5: SSOUR at 41 points, omega_L = 0.24825 on the LR sweep and
    # omega_R = 1.87087 on the RL sweep, 58 iterations
    n = 39
    d, b = W.laplace1d(n)
    pb = oracle.Problem(1, (n,), 3, d, (1,), library=L)
    x, exact, k = np.zeros(n), np.arange(1, n + 1) / 40, 0
    while k < 3000:
        x = pb.sor_sweep(oracle.DECOMPOSED, k, [0.24825, 1.87087], b, x)
        k += 1
        if np.abs(x - exact).sum() / 41 < 1e-3:
            break
    return k == 58


def pin_full_blocks(L):
    """Decomposed full ILU(0): L U = A on every subdomain block's pattern."""
    from tests.test_oracle_ilu_full import _block_lu, _blocks, _rand9
    n, sub = (11, 9), (3, 2)
    d = _rand9(n, 5)
    pb = oracle.Problem(2, n, 9, d, sub, library=L)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    F = pb.ilu0_export()
    nb = neighbours(full_n(n), 9)
    A = assemble(full_n(n), 9, d).toarray()
    for cells in _blocks(pb, n, sub).values():
        Lb, Ub = _block_lu(F, nb, cells)
        Ab = A[np.ix_(cells, cells)]
        if np.max(np.abs((Lb @ Ub - Ab)[Ab != 0])) > 1e-12 * np.max(np.abs(Ab)):
            return False
    return True


def pin_full_apply(L):
    """Decomposed full ILU(0) apply inverts (D + L') D^-1 (D + U')."""
    from tests.test_oracle_ilu_full import _rand9
    n, sub = (10, 9), (2, 3)
    pb = oracle.Problem(2, n, 9, _rand9(n, 8), sub, library=L)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    F = pb.ilu0_export()
    tf = pb.fwd_phase()
    fn = full_n(n)
    Lp = assemble(fn, 9, F, jmask_bool(pb.plan_info(1, tf)[0], 9), include_diag=False).toarray()
    Up = assemble(fn, 9, F, jmask_bool(pb.plan_info(1, tf ^ 1)[0], 9), include_diag=False).toarray()
    M = (np.diag(F[0]) + Lp) @ np.diag(1.0 / F[0]) @ (np.diag(F[0]) + Up)
    r = W.uniform_rhs(90, 3)
    return np.max(np.abs(M @ pb.ilu0_apply(r) - r)) <= 1e-12 * np.max(np.abs(r))


def pin_procedure(L):
    return procedure_holds((13, 11), (3, 2), L)


def pin_procedure3d(L):
    return procedure3d_holds((6, 5, 7), (2, 2, 3), L)


MUTANTS = [
    ("no interface coupling",
     "  return q_up_in_i && i_up_in_q;", "  return false;",
     [pin_table1_pgs2, pin_printed_systems, decomposed_within_table6, pin_procedure]),
    ("1D starts outward",
     "  if (d == 1) return (int)(t & 1);", "  if (d == 1) return (int)((t + 1) & 1);",
     [pin_table1_pgs2]),
    ("2D pair order swapped",
     "  int c = all ^ (tt >> 1);", "  int c = all ^ (tt >> 1) ^ ((tt >> 1) ? 3 : 0);",
     [pin_schedule, pin_printed_systems, pin_procedure]),
    ("sign of the old-value term",
     "      if (j >= 0) acc -= wi * aval(pb, k, i) * u[j];", "      if (j >= 0) acc += wi * aval(pb, k, i) * u[j];",
     [pin_splitting, pin_procedure]),
    ("dropped (1-w) D u term",
     "    double acc = (1.0 - wi) * aii * u[i] + wi * b[i];", "    double acc = wi * b[i];",
     [pin_splitting, pin_procedure]),
    ("transposed solve uses the row's own entry",
     "          coef = (scale ? scale[j] : 1.0) * ent(kb, j);",
     "          coef = (scale ? scale[i] : 1.0) * ent(k, i);",
     [pin_ssor_symmetric]),
    ("decomposed ILU uses a_ij twice",
     "          acc -= aval(pb, k, i) * aval(pb, kb, j) / pb.dtilde[j];",
     "          acc -= aval(pb, k, i) * aval(pb, k, i) / pb.dtilde[j];",
     [lambda L: pin_ilu_pattern(L, 1)]),
    ("natural ILU divides by the wrong pivot",
     "      L(ks[a], i) /= L(0, kc);", "      L(ks[a], i) /= L(0, i);",
     [lambda L: pin_ilu_pattern(L, 0)]),
    ("full ILU drops the update of later entries",
     "            F(ks[b2], i) -= lik * F(kk, kc);", "            (void)lik;",
     [pin_full_blocks]),
    ("full ILU stores l_ij instead of l_ij u_jj",
     "    for (int a = 0; a < nlow; ++a) F(ks[a], i) *= F(0, cols[a]);  // l_ij u_jj", "",
     [pin_full_blocks]),
    ("full ILU eliminates in the natural order in every subdomain",
     "      return precedes(ca, cb, cs);", "      return precedes(ca, cb, 0);",
     [pin_full_blocks]),
    ("full ILU apply solves the forward phase twice",
     "    return block_solve(pb, pbk, d.data(), nullptr, dy.data(), z, false, E);",
     "    return block_solve(pb, pf, d.data(), nullptr, dy.data(), z, false, E);",
     [pin_full_apply]),
    ("BiCGSTAB drops the omega step from x",
     "      for (int64_t i = 0; i < N; ++i) x[i] += alpha * ph[i] + om * sh[i];",
     "      for (int64_t i = 0; i < N; ++i) x[i] += alpha * ph[i];",
     [lambda L: pin_krylov_counts(L, "bicgstab")]),
    ("PCG beta from the wrong inner products",
     "      const double beta = rz2 / rz;", "      const double beta = rz / rz2;",
     [lambda L: pin_krylov_counts(L, "pcg")]),
    ("relaxation factor of the opposite direction",
     "    const double wi = omega[pl.corner[i]];", "    const double wi = omega[pl.corner[i] ^ 1];",
     [pin_table5_ssour, pin_procedure]),
    ("lexicographic order reversed",
     "    if (kq != ki) return kq < ki;", "    if (kq != ki) return kq > ki;",
     [pin_table1_pgs2, pin_printed_systems, pin_procedure]),
    ("9-point diagonal across an interface taken as new when upstream",
     "  if (nz != 1) return false;  // diagonal neighbour across an interface: old value",
     "  if (nz != 1) return precedes(cq, ci, csi);",
     [lambda L: face_sets_hold((13, 11), (3, 2), L), lambda L: reflected_blocks_hold((13, 11), (3, 2), L)]),
    ("column-wise order inside a subdomain (same iterate for 5 points, not for 9)",
     "  for (int a = 2; a >= 0; --a) {\n    int64_t kq", "  for (int a = 0; a < 3; ++a) {\n    int64_t kq",
     [lambda L: reflected_blocks_hold((13, 11), (3, 2), L)]),
    ("9-point D-ILU pivot sums the face neighbours only",
     "          if (pl.jmask[j] >> kb & 1) continue;  // mutual pair: no elimination term",
     "          if (pl.jmask[j] >> kb & 1) continue;  // mutual pair: no elimination term\n          if (k >= 5) continue;",
     [pin_dilu9]),
    ("3D neighbours along z sweep the same way",
     "  for (int a = 0; a < d; ++a)\n    if (idx[a] & 1) c ^= (1 << a);",
     "  for (int a = 0; a < d && a < 2; ++a)\n    if (idx[a] & 1) c ^= (1 << a);",
     [pin_procedure3d]),
]


def test_pins_hold_on_the_unmodified_oracle():
    L = oracle.lib()
    for _, _, _, pins in MUTANTS:
        for pin in pins:
            assert pin(L)


@pytest.mark.parametrize("name,anchor,replacement,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, anchor, replacement, pins):
    L = _build_mutant(tmp_path, anchor, replacement)
    assert not all(pin(L) for pin in pins), f"mistake not caught: {name}"
