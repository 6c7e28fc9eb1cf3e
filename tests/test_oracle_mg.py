"""Pins of the multigrid oracle (oracle/mg.py) against facts fixed outside it.

- the Galerkin product P^T A P against a dense product with a P built cell by
  cell, and against its closed form on the Poisson matrix;
- conservation: 1^T A_c 1 = 1^T A 1 (P 1 = 1);
- the coarsest level against the closed form of KC SSOR-Richardson steps,
  z = (I - (I - S A)^KC) A^-1 r;
- a two-level cycle against its dense error-propagation form
  I - B A = (I - S A)(I - ALPHA P B_c P^T A)(I - S A);
- symmetry and definiteness of B on a multi-level, multi-subdomain case;
- the smoother bound behind the omega < 1 reading: at omega = 1 the decomposed
  SSOR gives S A the eigenvalue d / (d - 2) = 2 on a 2 x 2 coupled corner block
  of the Poisson matrix (d = 4) and d / (d - 1) = 4/3 on a coupled pair.
"""
import types

import numpy as np
import pytest

import oracle
import oracle.mg as M
from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble


def _rand5(nx, ny, seed):
    """Random diagonally dominant 5-point entries (not symmetric)."""
    g = np.random.default_rng(seed)
    N = nx * ny
    d = -g.uniform(0.2, 1.0, size=(5, N))
    i = np.arange(N)
    x, y = i % nx, i // nx
    d[1][x == 0] = 0.0
    d[2][x == nx - 1] = 0.0
    d[3][y == 0] = 0.0
    d[4][y == ny - 1] = 0.0
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, size=N)
    return d


def _dense_P(nx, ny):
    nxc, nyc = (nx + 1) // 2, (ny + 1) // 2
    P = np.zeros((nx * ny, nxc * nyc))
    for y in range(ny):
        for x in range(nx):
            P[y * nx + x, (y // 2) * nxc + (x // 2)] = 1.0
    return P


def _dense(nx, ny, d):
    return assemble((nx, ny, 1), 5, d).toarray()


def _dense_op(fn, N):
    return np.stack([fn(e) for e in np.eye(N)], axis=1)


@pytest.mark.parametrize("nx,ny", [(7, 5), (8, 6), (9, 9), (2, 3), (1, 4)])
def test_galerkin_matches_dense_product(nx, ny):
    d = _rand5(nx, ny, nx * 10 + ny)
    P = _dense_P(nx, ny)
    C = P.T @ _dense(nx, ny, d) @ P
    dc = M.galerkin(nx, ny, d)
    nxc, nyc = (nx + 1) // 2, (ny + 1) // 2
    np.testing.assert_allclose(_dense(nxc, nyc, dc), C, rtol=0, atol=1e-13)


def test_galerkin_poisson_closed_form():
    # 2 x 2 aggregates of the 5-point Laplacian (4, -1): centre 4*4 - 2*4 = 8,
    # two unit couplings cross each aggregate side (-2); a one-cell-wide last
    # column (odd nx) holds 2 cells: centre 2*4 - 2 = 6, -2 to its west
    # aggregate, -1 across its south / north side.
    nx, ny = 9, 8
    dc = M.galerkin(nx, ny, W.poisson2d(nx, ny))
    nxc, nyc = 5, 4
    I = np.arange(nxc * nyc)
    X, Y = I % nxc, I // nxc
    last = X == nxc - 1
    np.testing.assert_array_equal(dc[0], np.where(last, 6.0, 8.0))
    np.testing.assert_array_equal(dc[1], np.where(X > 0, -2.0, 0.0))
    np.testing.assert_array_equal(dc[2], np.where(X < nxc - 1, -2.0, 0.0))
    np.testing.assert_array_equal(dc[3], np.where(Y > 0, np.where(last, -1.0, -2.0), 0.0))
    np.testing.assert_array_equal(dc[4], np.where(Y < nyc - 1, np.where(last, -1.0, -2.0), 0.0))


def test_galerkin_conserves_total():
    nx, ny = 33, 21
    d = _rand5(nx, ny, 5)
    dc = M.galerkin(nx, ny, d)
    assert abs(dc.sum() - d.sum()) <= 1e-12 * abs(d).sum()


def test_hierarchy_shape():
    H = M.Hierarchy(300, 260, W.poisson2d(300, 260), (3, 3), 0.9)
    assert [(nx, ny) for nx, ny, _ in H.levels] == [(300, 260), (150, 130), (75, 65), (38, 33), (19, 17)]
    assert [pb.sub[:2] for _, _, pb in H.levels] == [(3, 3), (9, 8), (4, 4), (2, 2), (1, 1)]
    assert len(M.Hierarchy(32, 20, W.poisson2d(32, 20), (2, 2), 0.9).levels) == 1


def test_coarsest_level_is_ssor_richardson():
    nx, ny, om = 24, 18, 0.9
    d = _rand5(nx, ny, 11)
    H = M.Hierarchy(nx, ny, d, (2, 3), om)
    assert len(H.levels) == 1
    N = nx * ny
    pb = H.levels[0][2]
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, om, e), N)
    A = _dense(nx, ny, d)
    E = np.linalg.matrix_power(np.eye(N) - S @ A, M.KC)
    r = np.random.default_rng(3).standard_normal(N)
    want = (np.eye(N) - E) @ np.linalg.solve(A, r)
    np.testing.assert_allclose(H.vcycle(r), want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_two_level_cycle_error_propagation():
    nx, ny, om = 40, 36, 0.85
    d = W.diffusion2d(W.loguniform_alpha(nx, ny, 9, 1.0, 10.0))
    H = M.Hierarchy(nx, ny, d, (2, 2), om)
    assert len(H.levels) == 2
    N = nx * ny
    pb, (nxc, nyc, pc) = H.levels[0][2], H.levels[1]
    Nc = nxc * nyc
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, om, e), N)
    Sc = _dense_op(lambda e: pc.ssor_apply(oracle.DECOMPOSED, om, e), Nc)
    A = _dense(nx, ny, d)
    P = _dense_P(nx, ny)
    Ac = P.T @ A @ P
    Bc = (np.eye(Nc) - np.linalg.matrix_power(np.eye(Nc) - Sc @ Ac, M.KC)) @ np.linalg.inv(Ac)
    I = np.eye(N)
    E = (I - S @ A) @ (I - M.ALPHA * P @ Bc @ P.T @ A) @ (I - S @ A)
    B = (I - E) @ np.linalg.inv(A)
    r = np.random.default_rng(4).standard_normal(N)
    want = B @ r
    np.testing.assert_allclose(H.vcycle(r), want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_cycle_symmetric_positive_definite():
    nx, ny = 150, 130
    d = W.diffusion2d(W.smoothed_lognormal_alpha(nx, ny, 21))
    H = M.Hierarchy(nx, ny, d, (3, 2), 0.9)
    assert len(H.levels) == 4
    g = np.random.default_rng(5)
    for _ in range(3):
        r1, r2 = g.standard_normal(nx * ny), g.standard_normal(nx * ny)
        a, b = H.vcycle(r1) @ r2, r1 @ H.vcycle(r2)
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
        assert H.vcycle(r1) @ r1 > 0


@pytest.mark.parametrize("sub,lam", [((3, 3), 2.0), ((1, 3), 4.0 / 3.0)])
def test_smoother_bound_at_omega_one(sub, lam):
    nx = 24
    N = nx * nx
    d = W.poisson2d(nx, nx)
    pb = oracle.Problem(2, (nx, nx), 5, d, sub)
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, 1.0, e), N)
    ev = np.linalg.eigvals(S @ _dense(nx, nx, d)).real
    assert abs(ev.max() - lam) < 1e-9
    S9 = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, 0.9, e), N)
    assert np.linalg.eigvals(S9 @ _dense(nx, nx, d)).real.max() < 2.0


def test_pcg_mg_converges_fast():
    nx = ny = 256
    d = W.diffusion2d(W.smoothed_lognormal_alpha(nx, ny, 31))
    b = W.uniform_rhs(nx * ny, 32)
    H = M.Hierarchy(nx, ny, d, (4, 4), 0.9)
    x, info = M.pcg(H, b, 1e-8, 200)
    assert info["status"] == 0 and info["iters"] <= 40
    r = b - H.levels[0][2].matvec(x)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)


# --- planted mistakes: each must fail at least one pin ------------------------

def _pin_galerkin(Mm):
    nx, ny = 7, 5
    d = _rand5(nx, ny, 75)
    P = _dense_P(nx, ny)
    try:
        dc = Mm.galerkin(nx, ny, d)
    except (ValueError, IndexError):
        return False
    return np.allclose(_dense(4, 3, dc), P.T @ _dense(nx, ny, d) @ P, rtol=0, atol=1e-13)


def _pin_coarsest(Mm):
    nx, ny, om = 12, 10, 0.9
    d = _rand5(nx, ny, 12)
    H = Mm.Hierarchy(nx, ny, d, (2, 2), om)
    N = nx * ny
    pb = H.levels[0][2]
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, om, e), N)
    A = _dense(nx, ny, d)
    r = np.random.default_rng(3).standard_normal(N)
    want = (np.eye(N) - np.linalg.matrix_power(np.eye(N) - S @ A, M.KC)) @ np.linalg.solve(A, r)
    return np.allclose(H.vcycle(r), want, rtol=0, atol=1e-11 * np.abs(want).max())


def _pin_two_level(Mm):
    nx, ny, om = 34, 30, 0.85
    d = _rand5(nx, ny, 34)
    H = Mm.Hierarchy(nx, ny, d, (2, 2), om)
    N = nx * ny
    pb = oracle.Problem(2, (nx, ny), 5, d, (2, 2))
    nxc, nyc = 17, 15
    P = _dense_P(nx, ny)
    A = _dense(nx, ny, d)
    Ac = P.T @ A @ P
    dc = np.zeros((5, nxc * nyc))
    for k, off in enumerate((0, -1, 1, -nxc, nxc)):
        for I in range(nxc * nyc):
            J = I + off
            if 0 <= J < nxc * nyc and (k < 1 or k > 2 or J // nxc == I // nxc):
                dc[k, I] = Ac[I, J]
    pc = oracle.Problem(2, (nxc, nyc), 5, dc, (1, 1))
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, om, e), N)
    Sc = _dense_op(lambda e: pc.ssor_apply(oracle.DECOMPOSED, om, e), nxc * nyc)
    Ic, I = np.eye(nxc * nyc), np.eye(N)
    Bc = (Ic - np.linalg.matrix_power(Ic - Sc @ Ac, M.KC)) @ np.linalg.inv(Ac)
    E = (I - S @ A) @ (I - M.ALPHA * P @ Bc @ P.T @ A) @ (I - S @ A)
    r = np.random.default_rng(4).standard_normal(N)
    want = (I - E) @ np.linalg.solve(A, r)
    try:
        got = H.vcycle(r)
    except (ValueError, IndexError):
        return False
    return len(H.levels) == 2 and np.allclose(got, want, rtol=0, atol=1e-10 * np.abs(want).max())


def _pin_galerkin3(Mm):
    n = (5, 4, 3)
    g = np.random.default_rng(53)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(7, N))
    d = W._zero_outside(d, n, 7)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, size=N)
    nx, ny, nz = n
    nc = [(v + 1) // 2 for v in n]
    P = np.zeros((N, nc[0] * nc[1] * nc[2]))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                P[(z * ny + y) * nx + x, ((z // 2) * nc[1] + y // 2) * nc[0] + x // 2] = 1.0
    try:
        dc = Mm.galerkin3(n, d)
    except (ValueError, IndexError):
        return False
    A = assemble(n, 7, d).toarray()
    return np.allclose(assemble(tuple(nc), 7, dc).toarray(), P.T @ A @ P, rtol=0, atol=1e-13)


MUTANTS = [
    ("        return z + self.smooth(k, r - pb.matvec(z))", "        return z"),
    ("P.T @ (r - pb.matvec(z))", "P.T @ (r + pb.matvec(z))"),
    ("ALPHA * (P @ self.vcycle(", "(P @ self.vcycle("),
    ("C = (P.T @ to_sparse(nx, ny, diags) @ P).tocoo()", "C = (P.T @ to_sparse(nx, ny, diags).T @ P).tocoo()"),
    ("    I = (y // 2) * nxc + x // 2", "    I = (x // 2) * nyc + y // 2"),
    ("            for _ in range(KC - 1):", "            for _ in range(KC):"),
    ("((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1))", "((0, 0), (1, 0), (-1, 0), (0, -1), (0, 1))"),
    ("        z = self.smooth(k, r)\n", "        z = 0.0 * r\n"),
    ("    I = ((z // 2) * nyc + y // 2) * nxc + x // 2", "    I = ((y // 2) * nzc + z // 2) * nxc + x // 2"),
    ("_OFF7 = ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))",
     "_OFF7 = ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, 1), (0, 0, -1))"),
]


def test_pins_hold_on_the_oracle():
    assert _pin_galerkin(M) and _pin_coarsest(M) and _pin_two_level(M) and _pin_galerkin3(M)


@pytest.mark.parametrize("anchor,replacement", MUTANTS)
def test_pins_catch_planted_mistake(anchor, replacement):
    src = open(M.__file__).read()
    assert src.count(anchor) == 1, anchor
    mod = types.ModuleType("mg_mutant")
    exec(compile(src.replace(anchor, replacement), "mg_mutant", "exec"), mod.__dict__)
    assert not (_pin_galerkin(mod) and _pin_coarsest(mod) and _pin_two_level(mod) and _pin_galerkin3(mod))


# --- 3D 7-point cycle ------------------------------------------------------------

def _rand7(n, seed):
    g = np.random.default_rng(seed)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(7, N))
    d = W._zero_outside(d, n, 7)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, size=N)
    return d


def _dense_P3(n):
    nx, ny, nz = n
    nc = [(v + 1) // 2 for v in n]
    P = np.zeros((nx * ny * nz, nc[0] * nc[1] * nc[2]))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                P[(z * ny + y) * nx + x, ((z // 2) * nc[1] + y // 2) * nc[0] + x // 2] = 1.0
    return P


def _dense3(n, d):
    return assemble(n, 7, d).toarray()


@pytest.mark.parametrize("n", [(5, 4, 3), (4, 4, 4), (3, 1, 5)])
def test_galerkin3_matches_dense_product(n):
    d = _rand7(n, sum(n))
    P = _dense_P3(n)
    nc = tuple((v + 1) // 2 for v in n)
    np.testing.assert_allclose(_dense3(nc, M.galerkin3(n, d)), P.T @ _dense3(n, d) @ P, rtol=0, atol=1e-13)


def test_galerkin3_poisson_closed_form():
    # 2 x 2 x 2 aggregates of the 7-point Laplacian (6, -1): centre 8*6 - 24 = 24,
    # four unit couplings cross each aggregate face (-4)
    n = (8, 6, 4)
    dc = M.galerkin3(n, W.poisson3d(*n))
    nc = (4, 3, 2)
    I = np.arange(np.prod(nc))
    X, Y, Z = I % nc[0], (I // nc[0]) % nc[1], I // (nc[0] * nc[1])
    np.testing.assert_array_equal(dc[0], np.full(I.size, 24.0))
    for k, (c, lim, sgn) in enumerate(((X, nc[0], -1), (X, nc[0], 1), (Y, nc[1], -1), (Y, nc[1], 1),
                                       (Z, nc[2], -1), (Z, nc[2], 1)), start=1):
        inside = (c > 0) if sgn < 0 else (c < lim - 1)
        np.testing.assert_array_equal(dc[k], np.where(inside, -4.0, 0.0))


def test_two_level_cycle3_error_propagation():
    n, om = (10, 8, 8), 0.85
    d = _rand7(n, 77)
    M.NMIN3, saved = 5, M.NMIN3  # two levels: 10 x 8 x 8 -> 5 x 4 x 4
    try:
        H = M.Hierarchy3(n, d, (2, 2, 2), om)
    finally:
        M.NMIN3 = saved
    assert len(H.levels) == 2
    N = int(np.prod(n))
    pb, (nc, _, pc) = H.levels[0][2], H.levels[1]
    Nc = int(np.prod(nc))
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, om, e), N)
    Sc = _dense_op(lambda e: pc.ssor_apply(oracle.DECOMPOSED, om, e), Nc)
    A = _dense3(n, d)
    P = _dense_P3(n)
    Ac = P.T @ A @ P
    Bc = (np.eye(Nc) - np.linalg.matrix_power(np.eye(Nc) - Sc @ Ac, M.KC)) @ np.linalg.inv(Ac)
    I = np.eye(N)
    E = (I - S @ A) @ (I - M.ALPHA * P @ Bc @ P.T @ A) @ (I - S @ A)
    r = np.random.default_rng(8).standard_normal(N)
    want = (I - E) @ np.linalg.solve(A, r)
    np.testing.assert_allclose(H.vcycle(r), want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_smoother3_bound_at_omega_one():
    # an interior vertex where eight subdomains start: the 2 x 2 x 2 corner block
    # of the 7-point Laplacian gives S A the eigenvalue 6 / (6 - 3) = 2
    n = (12, 12, 12)
    N = int(np.prod(n))
    d = W.poisson3d(*n)
    pb = oracle.Problem(3, n, 7, d, (3, 3, 3))
    A = _dense3(n, d)
    S = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, 1.0, e), N)
    assert abs(np.linalg.eigvals(S @ A).real.max() - 2.0) < 1e-9
    S9 = _dense_op(lambda e: pb.ssor_apply(oracle.DECOMPOSED, 0.9, e), N)
    assert np.linalg.eigvals(S9 @ A).real.max() < 2.0


def test_hierarchy3_shape_and_pcg():
    p = W.poisson3d_problem(48, 3)
    H = M.Hierarchy3(p["n"], p["diags"], p["sub"], 0.9)
    assert [lv[0] for lv in H.levels] == [(48, 48, 48), (24, 24, 24), (12, 12, 12)]
    assert [lv[2].sub for lv in H.levels] == [(3, 3, 3), (1, 1, 1), (1, 1, 1)]
    x, info = M.pcg(H, p["b"], 1e-8, 100)
    assert info["status"] == 0 and info["iters"] <= 20
