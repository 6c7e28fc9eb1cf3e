"""The oracle's implicit sets where the paper prints no system to check them
against, pinned to computations outside its own code.

9-point sweep (Sec. 3 extends the method to it without details):
- its implicit sets on the face neighbours are those of the 5-point sweep on
  the same grid and partition, which the printed coupled systems of Sec. 3-4
  pin; diagonal neighbours across an interface are never implicit;
- a 5-point matrix stored with zero corners sweeps exactly as the 5-point
  problem, coupled corner and edge blocks included;
- with the cross-interface face couplings zeroed (so no block carries a
  coupling), every subdomain's new values are the natural SOR sweep of its own
  block, cells in lexicographic order of the frame reflected along the axes it
  sweeps backwards, with every neighbour outside it (diagonal ones included)
  at its old value: a dense solve with numpy.

3D 7-point sweep (Sec. 4), all eight phases: the same per-subdomain reduction.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, neighbours
from tests.test_oracle_ilu_full import _parts

PARTS = [((13, 11), (3, 2)), ((9, 7), (9, 1)), ((16, 12), (2, 3)), ((10, 10), (1, 1)), ((12, 9), (4, 3)),
         ((7, 10), (1, 5))]


def _rand9(n, seed):
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.1, 1.0, size=(9, N))
    d = W._zero_outside(d, (n[0], n[1]), 9)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def _labels(n, sub):
    """Subdomain number of every cell."""
    lab = np.full(n[0] * n[1], -1, dtype=np.int64)
    idx = np.arange(n[0] * n[1])
    x, y = idx % n[0], idx // n[0]
    for s, (sx, sy) in enumerate(_parts(n, sub)):
        lab[np.isin(x, sx) & np.isin(y, sy)] = s
    assert (lab >= 0).all()
    return lab


def face_sets_hold(n, sub, library=None):
    """9-point face bits == 5-point bits; no diagonal bit across an interface."""
    p9 = oracle.Problem(2, n, 9, _rand9(n, 1), sub, library=library)
    p5 = oracle.Problem(2, n, 5, W.poisson2d(*n), sub, library=library)
    nb = neighbours(full_n(n), 9)
    lab = _labels(n, sub)
    faces = 0b11110
    for t in range(4):
        j9, c9, _, _ = p9.plan_info(oracle.DECOMPOSED, t)
        j5, c5, _, _ = p5.plan_info(oracle.DECOMPOSED, t)
        if not (np.array_equal(c9, c5) and np.array_equal(j9 & faces, j5 & faces)):
            return False
        for k in range(5, 9):
            across = (nb[k] >= 0) & (lab[np.maximum(nb[k], 0)] != lab)
            if ((j9[across] >> k) & 1).any():
                return False
    return True


def reflected_blocks_hold(n, sub, library=None):
    """With cross-interface face couplings zeroed, each subdomain's new values
    equal natural SOR of its block in reflected lexicographic order."""
    g = np.random.default_rng(31)
    N = n[0] * n[1]
    d = _rand9(n, 32)
    nb = neighbours(full_n(n), 9)
    lab = _labels(n, sub)
    for k in range(1, 5):
        across = (nb[k] >= 0) & (lab[np.maximum(nb[k], 0)] != lab)
        d[k, across] = 0.0
    pb = oracle.Problem(2, n, 9, d, sub, library=library)
    A = assemble(full_n(n), 9, d).toarray()
    omega = g.uniform(0.6, 1.8, size=4)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    idx = np.arange(N)
    x, y = idx % n[0], idx // n[0]
    for t in range(4):
        got = pb.sor_sweep(oracle.DECOMPOSED, t, omega, b, u)
        _, corner, _, _ = pb.plan_info(oracle.DECOMPOSED, t)
        for s in range(int(lab.max()) + 1):
            cells = idx[lab == s]
            cs = int(corner[cells[0]])
            if not (corner[cells] == cs).all():
                return False
            kx = -x[cells] if cs & 1 else x[cells]
            ky = -y[cells] if cs & 2 else y[cells]
            order = cells[np.lexsort((kx, ky))]
            out = idx[lab != s]
            As = A[np.ix_(order, order)]
            r = b[order] - A[np.ix_(order, out)] @ u[out]
            w = omega[cs]
            D = np.diag(np.diag(As))
            want = np.linalg.solve(D + w * np.tril(As, -1), ((1 - w) * D - w * np.triu(As, 1)) @ u[order] + w * r)
            if np.max(np.abs(got[order] - want)) > 1e-12 * np.max(np.abs(want)):
                return False
    return True


@pytest.mark.parametrize("n,sub", PARTS)
def test_face_sets_are_the_five_point_sets(orc, n, sub):
    assert face_sets_hold(n, sub)


@pytest.mark.parametrize("n,sub", PARTS)
@pytest.mark.parametrize("mode", [0, 1])
def test_five_point_matrix_in_nine_point_storage_sweeps_as_five_point(orc, n, sub, mode):
    g = np.random.default_rng(21)
    N = n[0] * n[1]
    d5 = W.diffusion2d(W.smoothed_lognormal_alpha(n[0], n[1], 22))
    p5 = orc.Problem(2, n, 5, d5, sub)
    p9 = orc.Problem(2, n, 9, W.embed5in9(d5), sub)
    omega = g.uniform(0.6, 1.8, size=4)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    for t in range(4):
        x5 = p5.sor_sweep(mode, t, omega, b, u)
        x9 = p9.sor_sweep(mode, t, omega, b, u)
        assert np.max(np.abs(x9 - x5)) <= 1e-14 * np.max(np.abs(x5)), t


@pytest.mark.parametrize("n,sub", PARTS)
def test_subdomain_sweep_is_natural_sor_of_its_reflected_block(orc, n, sub):
    assert reflected_blocks_hold(n, sub)


def _labels3(n, sub):
    """Subdomain number of every cell of a 3D grid (equal split, the first
    n mod p parts one longer)."""
    cuts = []
    for a in range(3):
        q, r = divmod(n[a], sub[a])
        cuts.append(np.repeat(np.arange(sub[a]), [q + (1 if k < r else 0) for k in range(sub[a])]))
    N = n[0] * n[1] * n[2]
    idx = np.arange(N)
    x, y, z = idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])
    return cuts[0][x] + sub[0] * (cuts[1][y] + sub[1] * cuts[2][z]), (x, y, z)


@pytest.mark.parametrize("n,sub", [((6, 5, 7), (2, 2, 3)), ((5, 4, 6), (5, 1, 2)), ((4, 6, 5), (1, 1, 1))])
def test_3d_subdomain_sweep_is_natural_sor_of_its_reflected_block(orc, n, sub):
    # Sec. 4: each subdomain sweeps from its start corner; with every coupling
    # across an interface removed, its new values are natural (lexicographic
    # z, y, x) SOR of its block in the frame reflected along the axes it
    # sweeps backwards, with outside neighbours at their old values.
    g = np.random.default_rng(41)
    N = int(np.prod(n))
    lab, (x, y, z) = _labels3(n, sub)
    d = -g.uniform(0.1, 1.0, size=(7, N))
    nb = neighbours(n, 7)
    d[nb < 0] = 0.0
    for k in range(1, 7):
        across = (nb[k] >= 0) & (lab[np.maximum(nb[k], 0)] != lab)
        d[k, across] = 0.0
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    pb = orc.Problem(3, n, 7, d, sub)
    A = assemble(n, 7, d).toarray()
    omega = g.uniform(0.6, 1.8, size=8)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    idx = np.arange(N)
    for t in range(8):
        got = pb.sor_sweep(orc.DECOMPOSED, t, omega, b, u)
        _, corner, _, _ = pb.plan_info(orc.DECOMPOSED, t)
        for s in np.unique(lab):
            cells = idx[lab == s]
            cs = int(corner[cells[0]])
            assert (corner[cells] == cs).all()
            keys = [-c[cells] if cs >> a & 1 else c[cells] for a, c in enumerate((x, y, z))]
            order = cells[np.lexsort(keys)]
            out = idx[lab != s]
            As = A[np.ix_(order, order)]
            r = b[order] - A[np.ix_(order, out)] @ u[out]
            w = omega[cs]
            D = np.diag(np.diag(As))
            want = np.linalg.solve(D + w * np.tril(As, -1), ((1 - w) * D - w * np.triu(As, 1)) @ u[order] + w * r)
            assert np.max(np.abs(got[order] - want)) <= 1e-12 * np.max(np.abs(want)), (t, s)
