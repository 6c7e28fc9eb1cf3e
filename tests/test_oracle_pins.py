"""Pins of the CPU oracle against the paper and against mathematics that do not
depend on the oracle's own code (closed forms, library solves, the paper's
printed coupled systems and schedule)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, jmask_bool, neighbours

NE, NW, SE, SW = 3, 2, 1, 0  # start corner bits (x: 1 = starts at max x, y: 2)


def _random_diags(n, stencil, seed, symmetric=False):
    """Strictly diagonally dominant n-diagonal matrix with random entries."""
    g = np.random.default_rng(seed)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(stencil, N))
    nb = neighbours(full_n(n), stencil)
    d[nb < 0] = 0.0
    if symmetric:
        opp = {1: 2, 3: 4, 5: 6}
        for k, ko in opp.items():
            if k < stencil and ko < stencil:
                ok = nb[k] >= 0
                d[k, ok] = d[ko, nb[k][ok]]
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, size=N)
    return d


def _cell(n, x, y, z=0):
    return x + n[0] * (y + n[1] * z)


# ---------------------------------------------------------------------------
# Schedule (Sec. 2 step (ii); Sec. 3 example and "Sweeping directions"; Sec. 4)
# ---------------------------------------------------------------------------

def test_schedule_2d_matches_paper_example(orc):
    # 2x2 subdomains numbered 1..4 = (0,0), (1,0), (0,1), (1,1): first sweep
    # NE, NW, SE, SW; next sweep the opposite directions SW, SE, NW, NE; then a
    # new diagonal (SE-NW) for the next pair of sweeps.
    n = (6, 6, 1)
    pb = orc.Problem(2, n, 5, W.poisson2d(6, 6), (2, 2))
    centres = [_cell(n, 1, 1), _cell(n, 4, 1), _cell(n, 1, 4), _cell(n, 4, 4)]
    want = {0: [NE, NW, SE, SW], 1: [SW, SE, NW, NE]}
    for t, w in want.items():
        _, corner, _, _ = pb.plan_info(orc.DECOMPOSED, t)
        assert [int(corner[c]) for c in centres] == w
    _, c0, _, _ = pb.plan_info(orc.DECOMPOSED, 0)
    _, c2, _, _ = pb.plan_info(orc.DECOMPOSED, 2)
    _, c3, _, _ = pb.plan_info(orc.DECOMPOSED, 3)
    assert int(c2[centres[0]]) == NW  # Omega_1 moves from SW-NE to SE-NW
    for c in centres:
        # every subdomain takes the other diagonal, reversed within the pair
        assert {int(c2[c]), int(c3[c])} == {int(c0[c]) ^ 1, int(c0[c]) ^ 2}
        assert int(c2[c]) ^ int(c3[c]) == 3


@pytest.mark.parametrize("dim,sub", [(1, (5,)), (2, (4, 3)), (2, (5, 1)), (3, (3, 2, 2))])
def test_schedule_rules_hold_for_every_phase(orc, dim, sub):
    # neighbours along an axis sweep opposite along it; all directions reverse
    # every sweep; each subdomain visits all 2^d corners in 2^d sweeps.
    for t in range(2 ** dim):
        cs = {}
        for idx in np.ndindex(*sub):
            c = orc.base_corner(dim, t)
            for a in range(dim):
                if idx[a] & 1:
                    c ^= 1 << a
            cs[idx] = c
        for idx, c in cs.items():
            for a in range(dim):
                j = list(idx); j[a] += 1
                if j[a] < sub[a]:
                    assert (c ^ cs[tuple(j)]) >> a & 1
        cnext = orc.base_corner(dim, t + 1)
        assert orc.base_corner(dim, t) ^ cnext == (1 << dim) - 1 or (t % 2 == 1)
        if t % 2 == 0:
            assert orc.base_corner(dim, t) ^ cnext == (1 << dim) - 1
    assert sorted(orc.base_corner(dim, t) for t in range(2 ** dim)) == list(range(2 ** dim))


# ---------------------------------------------------------------------------
# Coupled systems (Eqs. 1d:sorc, 2d:sor4b4, 2d:sor2b2; Sec. 4)
# ---------------------------------------------------------------------------
W_, E_, S_, N_, B_, F_ = 1, 2, 3, 4, 5, 6


def _J(jm, c):
    return {k for k in range(1, 9) if (int(jm[c]) >> k) & 1}


def test_1d_start_nodes_form_the_2x2_system(orc):
    # Eq. (1d:sorc): when both subdomains start at the interface, u_m and
    # u_{m+1} are solved together from old u_{m-1}, u_{m+2}.
    n = 10
    d, _ = W.laplace1d(n)
    pb = orc.Problem(1, (n,), 3, d, (2,))
    jm, _, nb, mb = pb.plan_info(orc.DECOMPOSED, 1)
    assert mb == 2 and nb == n - 1
    assert _J(jm, 4) == {E_} and _J(jm, 5) == {W_}
    jm0, _, _, mb0 = pb.plan_info(orc.DECOMPOSED, 0)
    assert mb0 == 1  # the first sweep runs towards the interface: no system


def test_2d_corner_and_edge_systems_match_the_printed_equations(orc):
    # 6x6 grid, 2x2 subdomains, first sweep. Node #1 of Omega_1 is (i,j)=(2,2).
    n = (6, 6, 1)
    pb = orc.Problem(2, n, 5, W.poisson2d(6, 6), (2, 2))
    jm, _, nblocks, mb = pb.plan_info(orc.DECOMPOSED, 0)
    # Eq. (2d:sor4b4): row 1 (NE) new E, N; row 2 (NW) new W, N; row 3 (SE)
    # new S, E; row 4 (SW) new S, W; all other neighbours old.
    assert _J(jm, _cell(n, 2, 2)) == {E_, N_}
    assert _J(jm, _cell(n, 3, 2)) == {W_, N_}
    assert _J(jm, _cell(n, 2, 3)) == {S_, E_}
    assert _J(jm, _cell(n, 3, 3)) == {S_, W_}
    # Eq. (2d:sor2b2): u_{i-1,j} (NE) uses new u_{i,j} (E) and is coupled to
    # u_{i-1,j+1} (N); u_{i-1,j+1} (SE) uses new u_{i,j+1} (E) and u_{i-1,j} (S).
    assert _J(jm, _cell(n, 1, 2)) == {E_, N_}
    assert _J(jm, _cell(n, 1, 3)) == {E_, S_}
    assert mb == 4
    # one 4x4 corner system, 4 edges x 2 pairs, 36 - 4 - 16 singletons
    assert nblocks == 1 + 8 + (36 - 4 - 16)
    # next sweep (opposite directions): "no need to solve local systems"
    _, _, nb1, mb1 = pb.plan_info(orc.DECOMPOSED, 1)
    assert mb1 == 1 and nb1 == 36


def test_3d_corner_edge_face_systems(orc):
    # Sec. 4: an 8x8 corner system with 32 nonzeros, 4x4 systems along the
    # three coupling edges, 2x2 systems on the three coupling faces.
    m = 6
    pb = orc.Problem(3, (m, m, m), 7, W.poisson3d(m, m, m), (2, 2, 2))
    jm, _, nblocks, mb = pb.plan_info(orc.DECOMPOSED, 0)
    assert mb == 8
    corner = [_cell((m, m, m), x, y, z) for x in (2, 3) for y in (2, 3) for z in (2, 3)]
    nnz = 8 + sum(len(_J(jm, c)) for c in corner)
    assert nnz == 32
    n8 = 1
    n4 = 3 * 2 * 2          # 3 edge lines, 2 halves, 2 positions beyond the corner
    n2 = 3 * 4 * 2 * 2      # 3 planes, 4 quadrants, 2 x 2 positions
    assert nblocks == n8 + n4 + n2 + (m ** 3 - 8 - 4 * n4 - 2 * n2)


# ---------------------------------------------------------------------------
# One sweep == its splitting equation, solved by a library sparse solver
# (Eq. ca2d:matiter: (D + w L_J) u+ = ((1-w) D - w U_J) u + w b)
# ---------------------------------------------------------------------------
CASES = [
    (1, (23,), 3, (3,)),
    (2, (13, 11), 5, (2, 2)),
    (2, (17, 9), 5, (3, 2)),
    (2, (16, 7), 5, (4, 1)),
    (2, (9, 12), 9, (2, 3)),
    (3, (7, 6, 5), 7, (2, 2, 2)),
    (3, (8, 5, 6), 7, (3, 1, 2)),
]


@pytest.mark.parametrize("dim,n,stencil,sub", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_sweep_solves_the_splitting_equation(orc, dim, n, stencil, sub, mode):
    g = np.random.default_rng(7)
    fn = full_n(n)
    N = int(np.prod(fn))
    d = _random_diags(fn, stencil, 3)
    pb = orc.Problem(dim, n, stencil, d, sub)
    omega = g.uniform(0.6, 1.8, size=2 ** dim)
    b = g.uniform(-1, 1, N)
    u = g.uniform(-1, 1, N)
    for t in range(2 ** dim):
        x = pb.sor_sweep(mode, t, omega, b, u)
        jm, corner, _, _ = pb.plan_info(mode, t)
        J = jmask_bool(jm, stencil)
        nb = neighbours(fn, stencil)
        U = ~J & (nb >= 0)
        U[0] = False
        w = omega[corner] if mode == 1 else np.full(N, omega[0])
        L = assemble(fn, stencil, d, J, include_diag=False)
        Um = assemble(fn, stencil, d, U, include_diag=False)
        D = sp.diags(d[0])
        Wd = sp.diags(w)
        lhs = (D + Wd @ L).tocsc()
        rhs = (sp.diags(1 - w) @ D - Wd @ Um) @ u + w * b
        ref = spla.spsolve(lhs, rhs)
        assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim,n,stencil", [(2, (11, 9), 5), (3, (5, 6, 4), 7), (2, (8, 10), 9), (1, (17,), 3)])
def test_one_subdomain_equals_natural_order(orc, dim, n, stencil):
    fn = full_n(n)
    d = _random_diags(fn, stencil, 11)
    N = int(np.prod(fn))
    g = np.random.default_rng(3)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    pb = orc.Problem(dim, n, stencil, d, (1, 1, 1))
    t0 = orc.lib().orc_fwd_phase(dim)  # phase whose start corner is the origin
    assert orc.base_corner(dim, t0) == 0
    for om in (1.0, 1.37):
        x_dec = pb.sor_sweep(orc.DECOMPOSED, t0, om, b, u)
        x_nat = pb.sor_sweep(orc.NATURAL, 0, om, b, u)
        assert np.array_equal(x_dec, x_nat)
        # natural SOR = (D + w tril(A,-1)) x = ((1-w) D - w triu(A,1)) u + w b
        A = assemble(fn, stencil, d).toarray()
        Dm = np.diag(np.diag(A))
        ref = np.linalg.solve(Dm + om * np.tril(A, -1), ((1 - om) * Dm - om * np.triu(A, 1)) @ u + om * b)
        assert np.max(np.abs(x_nat - ref)) <= 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Closed-form contraction rates on the Poisson model (Young's theory)
# ---------------------------------------------------------------------------

def _late_contraction(orc, pb, mode, omega, n, sweeps, tail, phase=lambda k: 0):
    g = np.random.default_rng(5)
    N = n * n
    x = g.uniform(-1, 1, N)
    b = np.zeros(N)
    norms = []
    for k in range(sweeps):
        x = pb.sor_sweep(mode, phase(k), omega, b, x)
        norms.append(np.linalg.norm(x))
    return (norms[-1] / norms[-1 - tail]) ** (1.0 / tail)


@pytest.mark.parametrize("omega", [1.0, 1.5, 1.7])
def test_natural_sor_rate_matches_young_formula(orc, omega):
    n = 24
    pb = orc.Problem(2, (n, n), 5, W.poisson2d(n, n), (1, 1))
    mu = math.cos(math.pi / (n + 1))
    wopt = 2.0 / (1.0 + math.sin(math.pi / (n + 1)))
    assert omega < wopt
    rho = ((omega * mu + math.sqrt(omega ** 2 * mu ** 2 - 4 * (omega - 1))) / 2) ** 2
    got = _late_contraction(orc, pb, orc.NATURAL, omega, n, 1500, 200)
    assert abs(got - rho) <= 2e-3 * rho


def test_gauss_seidel_rate_is_cos_squared(orc):
    n = 20
    pb = orc.Problem(2, (n, n), 5, W.poisson2d(n, n), (1, 1))
    got = _late_contraction(orc, pb, orc.NATURAL, 1.0, n, 1500, 200)
    assert abs(got - math.cos(math.pi / (n + 1)) ** 2) <= 1e-4


def test_sor_at_optimal_omega_contracts_at_omega_minus_one(orc):
    # At w_opt the iteration matrix has a Jordan block, so the observed
    # contraction approaches w-1 from above slowly: 2 % slack on 64 x 64.
    n = 64
    wopt = 2.0 / (1.0 + math.sin(math.pi / (n + 1)))
    pb = orc.Problem(2, (n, n), 5, W.poisson2d(n, n), (1, 1))
    got = _late_contraction(orc, pb, orc.NATURAL, wopt, n, 700, 100)
    assert (wopt - 1) <= got <= (wopt - 1) * 1.02


def test_theorem1_condition_gives_convergence_in_1d(orc):
    # Theorem 1: |1 - w_L| |1 - w_R| < 1 suffices; w_L = 0.2, w_R = 1.9.
    n = 60
    d, b = W.laplace1d(n)
    pb = orc.Problem(1, (n,), 3, d, (4,))
    x = np.zeros(n)
    for k in range(4000):
        x = pb.sor_sweep(orc.DECOMPOSED, k, [0.2, 1.9], b, x)
    assert np.max(np.abs(x - np.arange(1, n + 1) / (n + 1))) < 1e-8


def test_theorem2_condition_gives_convergence_in_2d(orc):
    n = 16
    pb = orc.Problem(2, (n, n), 5, W.poisson2d(n, n), (3, 2))
    omega = [0.3, 1.95, 1.0, 1.7]  # product of |1 - w| = 0.7*0.95*0*0.7 < 1
    b = W.uniform_rhs(n * n, 1)
    x = np.zeros(n * n)
    for k in range(3000):
        x = pb.sor_sweep(orc.DECOMPOSED, k, omega, b, x)
    A = assemble((n, n, 1), 5, W.poisson2d(n, n)).toarray()
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Solvers agree with a dense direct solve on tiny grids
# ---------------------------------------------------------------------------
SOLVE_CASES = [
    ("pcg", "ssor", 1, 2, (12, 10), 5, (2, 3), True),
    ("pcg", "none", 1, 2, (12, 10), 5, (2, 3), True),
    ("pcg", "ssor", 0, 3, (6, 5, 4), 7, (1, 1, 1), True),
    ("pcg", "ssor", 1, 3, (6, 5, 4), 7, (2, 2, 2), True),
    ("bicgstab", "ilu0", 1, 2, (12, 10), 5, (3, 2), False),
    ("bicgstab", "ilu0", 0, 2, (12, 10), 5, (1, 1), False),
    ("bicgstab", "ilu0", 1, 3, (6, 5, 4), 7, (2, 2, 2), False),
    ("bicgstab", "ilu0", 0, 2, (10, 10), 9, (1, 1), False),
    ("bicgstab", "ilu0", 1, 2, (10, 10), 9, (2, 2), False),
    ("stationary", "none", 1, 2, (12, 10), 5, (2, 3), False),
    ("stationary", "none", 1, 3, (6, 5, 4), 7, (2, 2, 2), False),
]


@pytest.mark.parametrize("method,prec,mode,dim,n,stencil,sub,sym", SOLVE_CASES)
def test_solvers_agree_with_dense_direct_solve(orc, method, prec, mode, dim, n, stencil, sub, sym):
    fn = full_n(n)
    N = int(np.prod(fn))
    d = _random_diags(fn, stencil, 21, symmetric=sym)
    b = W.uniform_rhs(N, 4)
    pb = orc.Problem(dim, n, stencil, d, sub)
    M = {"pcg": orc.PCG, "bicgstab": orc.BICGSTAB, "stationary": orc.STATIONARY}[method]
    P = {"none": orc.PREC_NONE, "ssor": orc.PREC_SSOR, "ilu0": orc.PREC_ILU0}[prec]
    x, info = pb.solve(M, P, mode, 1.2 if method == "stationary" else 1.0, 1e-12, 20000, b)
    A = assemble(fn, stencil, d).toarray()
    ref = np.linalg.solve(A, b)
    assert info["status"] == 0 and info["relres"] <= 1e-12
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def krylov_counts_match_scipy(L, method):
    """Iteration counts of the oracle's PCG / BiCGSTAB against scipy's
    implementations of the same algorithms with the same preconditioner
    (scipy counts the early exit on ||s|| one iteration less)."""
    import oracle
    n, N = (20, 17, 1), 340
    b = W.uniform_rhs(N, 4)
    if method == "bicgstab":
        d = _random_diags(n, 5, 21)
        pb = oracle.Problem(2, n, 5, d, (2, 3), library=L)
        pb.ilu0_factor(oracle.DECOMPOSED)
        _, info = pb.solve(oracle.BICGSTAB, oracle.PREC_ILU0, 1, 1.0, 1e-10, 300, b)
        Mop = lambda r: pb.ilu0_apply(r)
        solver = spla.bicgstab
    else:
        d = W.diffusion2d(W.loguniform_alpha(20, 17, 3))
        pb = oracle.Problem(2, n, 5, d, (2, 3), library=L)
        _, info = pb.solve(oracle.PCG, oracle.PREC_SSOR, 1, 1.0, 1e-10, 500, b)
        Mop = lambda r: pb.ssor_apply(oracle.DECOMPOSED, 1.0, r)
        solver = spla.cg
    cnt = [0]
    _, flag = solver(assemble(n, 5, d).tocsr(), b, rtol=1e-10, atol=0,
                     M=spla.LinearOperator((N, N), matvec=Mop), maxiter=500,
                     callback=lambda xk: cnt.__setitem__(0, cnt[0] + 1))
    return flag == 0 and info["status"] == 0 and abs(info["iters"] - cnt[0]) <= 1


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_krylov_iteration_counts_match_scipy(orc, method):
    assert krylov_counts_match_scipy(orc.lib(), method)


# ---------------------------------------------------------------------------
# ILU(0) (Sec. 5): (LU)_ij = A_ij on the pattern
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,stencil", [(2, (9, 7), 5), (3, (5, 4, 6), 7), (2, (8, 9), 9)])
def test_natural_ilu0_reproduces_A_on_its_pattern(orc, dim, n, stencil):
    fn = full_n(n)
    d = _random_diags(fn, stencil, 31)
    pb = orc.Problem(dim, n, stencil, d, (1, 1, 1))
    pb.ilu0_factor(orc.NATURAL)
    f = pb.ilu0_export()
    nb = neighbours(fn, stencil)
    N = nb.shape[1]
    idx = np.arange(N)
    lower = (nb >= 0) & (nb < idx)
    upper = (nb > idx)
    L = assemble(fn, stencil, f, lower, include_diag=False).toarray() + np.eye(N)
    U = assemble(fn, stencil, f, upper, include_diag=True).toarray()
    A = assemble(fn, stencil, d).toarray()
    LU = L @ U
    pat = A != 0
    assert np.max(np.abs((LU - A)[pat])) <= 1e-12 * np.max(np.abs(A))
    r = W.uniform_rhs(N, 9)
    assert np.allclose(LU @ pb.ilu0_apply(r), r, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim,n,stencil,sub", [(2, (13, 11), 5, (3, 2)), (3, (6, 7, 5), 7, (2, 3, 2)),
                                               (2, (12, 10), 5, (1, 1))])
def test_decomposed_ilu0_reproduces_A_on_its_pattern(orc, dim, n, stencil, sub):
    fn = full_n(n)
    d = _random_diags(fn, stencil, 41)
    N = int(np.prod(fn))
    pb = orc.Problem(dim, n, stencil, d, sub)
    pb.ilu0_factor(orc.DECOMPOSED)
    dt = pb.ilu0_export()
    tf = pb.fwd_phase()
    jf, _, _, _ = pb.plan_info(orc.DECOMPOSED, tf)
    jb, _, _, _ = pb.plan_info(orc.DECOMPOSED, tf ^ 1)
    Jf, Jb = jmask_bool(jf, stencil), jmask_bool(jb, stencil)
    nb = neighbours(fn, stencil)
    # the reverse phase's implicit set is exactly the complement (5/7-point)
    assert np.array_equal(Jb[1:], ~Jf[1:] & (nb[1:] >= 0))
    Lj = assemble(fn, stencil, d, Jf, include_diag=False).toarray()
    Uj = assemble(fn, stencil, d, Jb, include_diag=False).toarray()
    Dt = np.diag(dt)
    M = (Dt + Lj) @ np.diag(1 / dt) @ (Dt + Uj)
    A = assemble(fn, stencil, d).toarray()
    pat = A != 0
    assert np.max(np.abs((M - A)[pat])) <= 1e-12 * np.max(np.abs(A))
    r = W.uniform_rhs(N, 8)
    assert np.allclose(M @ pb.ilu0_apply(r), r, rtol=0, atol=1e-11)
    if sub == (1, 1):
        pn = orc.Problem(dim, n, stencil, d, sub)
        pn.ilu0_factor(orc.NATURAL)
        assert np.allclose(pn.ilu0_export()[0], dt, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n,sub", [((10, 9), (2, 2)), ((13, 11), (3, 2)), ((9, 7), (9, 1)), ((12, 9), (4, 3)),
                                   ((7, 10), (1, 5)), ((10, 10), (1, 1))])
def test_decomposed_ilu0_9pt_is_dilu(orc, n, sub):
    # Reading 12 keeps A's off-diagonals in L and U and chooses the pivots so
    # that M = (D~ + L) D~^-1 (D~ + U) has A's diagonal: the definition of
    # D-ILU, which fixes every pivot once the upstream sets are fixed (those
    # are pinned in test_oracle_sweep_sets.py). Also M z = r for the apply.
    fn = full_n(n)
    N = int(np.prod(fn))
    d = _random_diags(fn, 9, 51)
    pb = orc.Problem(2, n, 9, d, sub)
    pb.ilu0_factor(orc.DECOMPOSED)
    dt = pb.ilu0_export()
    tf = pb.fwd_phase()
    Jf = jmask_bool(pb.plan_info(orc.DECOMPOSED, tf)[0], 9)
    Jb = jmask_bool(pb.plan_info(orc.DECOMPOSED, tf ^ 1)[0], 9)
    Lj = assemble(fn, 9, d, Jf, include_diag=False).toarray()
    Uj = assemble(fn, 9, d, Jb, include_diag=False).toarray()
    M = (np.diag(dt) + Lj) @ np.diag(1 / dt) @ (np.diag(dt) + Uj)
    A = assemble(fn, 9, d).toarray()
    assert np.max(np.abs(np.diag(M) - np.diag(A))) <= 1e-14 * np.max(np.abs(np.diag(A)))
    r = W.uniform_rhs(N, 2)
    assert np.allclose(M @ pb.ilu0_apply(r), r, rtol=0, atol=1e-11)


# ---------------------------------------------------------------------------
# SSOR apply: symmetric positive definite, classical SSOR with one subdomain
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,stencil,sub", [(2, (11, 9), 5, (2, 3)), (3, (5, 6, 4), 7, (2, 2, 2)),
                                               (2, (9, 8), 9, (2, 2)), (2, (9, 8), 5, (1, 1))])
def test_ssor_apply_is_the_symmetric_closed_form(orc, dim, n, stencil, sub):
    fn = full_n(n)
    N = int(np.prod(fn))
    d = _random_diags(fn, stencil, 61)  # nonsymmetric A: M must still be symmetric
    pb = orc.Problem(dim, n, stencil, d, sub)
    om = 1.3
    g = np.random.default_rng(2)
    r1, r2 = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    z1, z2 = pb.ssor_apply(orc.DECOMPOSED, om, r1), pb.ssor_apply(orc.DECOMPOSED, om, r2)
    assert abs(z1 @ r2 - z2 @ r1) <= 1e-13 * np.linalg.norm(z1) * np.linalg.norm(r2)
    assert z1 @ r1 > 0 and z2 @ r2 > 0
    Jf = jmask_bool(pb.plan_info(orc.DECOMPOSED, pb.fwd_phase())[0], stencil)
    L = assemble(fn, stencil, d, Jf, include_diag=False).toarray()
    D = np.diag(d[0])
    M = (D + om * L) @ np.diag(1 / d[0]) @ (D + om * L).T / (om * (2 - om))
    assert np.allclose(M @ z1, r1, rtol=0, atol=1e-11)
    if sub == (1, 1):
        A = assemble(fn, stencil, d).toarray()
        Ml = (D + om * np.tril(A, -1)) @ np.diag(1 / d[0]) @ (D + om * np.tril(A, -1)).T / (om * (2 - om))
        assert np.allclose(Ml @ z1, r1, rtol=0, atol=1e-11)
