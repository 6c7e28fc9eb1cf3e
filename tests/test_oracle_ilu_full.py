"""The oracle's decomposed full ILU(0) (Sec. 5 with the reading that within
every subdomain the factor is the ILU(0) of A's diagonal block in that
subdomain's own order, and that across interfaces the couplings are those of
the decomposed sweep) pinned to textbook computations:

- with one subdomain it is the natural IKJ ILU(0), bit for bit;
- on every subdomain block, (L U)_ij = A_ij on the block's pattern, with L and
  U supported on that pattern (the defining property of ILU(0));
- a 5-point matrix stored with zero corners gets, block by block, the textbook
  level-of-fill ILU(1) (Saad Alg. 10.5) of the block in its sweep order: the
  decomposed ILU(1);
- on 5-point matrices it is the decomposed ILU(0);
- its apply inverts M = (D + L') D^-1 (D + U') assembled from the factor and
  the implicit sets of the forward phase and its reverse.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, jmask_bool, neighbours
from tests.test_oracle_iluk import _iluk_dense, _rand5


def _rand9(n, seed):
    """Diagonally dominant nonsymmetric 9-point matrix, zero outside the grid."""
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.1, 1.0, size=(9, N))
    d = W._zero_outside(d, (n[0], n[1]), 9)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def _blocks(pb, n, sub):
    """Cells of every subdomain, each in its own forward-phase sweep order
    (lexicographic in the frame reflected along the axes it sweeps backwards)."""
    _, corner, _, _ = pb.plan_info(oracle.DECOMPOSED, pb.fwd_phase())
    nx, ny = n
    idx = np.arange(nx * ny)
    x, y = idx % nx, idx // nx
    out = {}
    for sx, sy in _parts(n, sub):
        cells = idx[np.isin(x, sx) & np.isin(y, sy)]
        cs = int(corner[cells[0]])
        kx = -x[cells] if cs & 1 else x[cells]
        ky = -y[cells] if cs & 2 else y[cells]
        out[(sx[0], sy[0])] = cells[np.lexsort((kx, ky))]
    return out


def _parts(n, sub):
    """Equal split, the first n mod p parts one longer (as the oracle splits)."""
    res = []
    splits = []
    for a in range(2):
        p, m = sub[a], n[a]
        q, r = divmod(m, p)
        lo = [k * q + min(k, r) for k in range(p)]
        splits.append([np.arange(lo[k], lo[k] + q + (1 if k < r else 0)) for k in range(p)])
    for sy in splits[1]:
        for sx in splits[0]:
            res.append((sx, sy))
    return res


def _block_lu(F, nb, cells):
    """Unit-lower L and upper U of one block from the full factor F
    (lower entries l_ij u_jj, upper u_ij) in the block's order."""
    m = len(cells)
    pos = {int(c): p for p, c in enumerate(cells)}
    L, U = np.eye(m), np.zeros((m, m))
    for p, i in enumerate(cells):
        U[p, p] = F[0, i]
        for k in range(1, F.shape[0]):
            j = nb[k, i]
            if j < 0 or int(j) not in pos:
                continue
            q = pos[int(j)]
            if q < p:
                L[p, q] = F[k, i] / F[0, j]
            else:
                U[p, q] = F[k, i]
    return L, U


@pytest.mark.parametrize("n", [(9, 7), (6, 11)])
def test_one_subdomain_is_the_natural_factor(n):
    d = _rand9(n, 3 + n[0])
    nat = oracle.Problem(2, n, 9, d, (1, 1))
    nat.ilu0_factor(oracle.NATURAL)
    f = nat.ilu0_export()  # lower entries l_ij, upper u_ij
    nb = neighbours(full_n(n), 9)
    idx = np.arange(n[0] * n[1])
    want = f.copy()
    for k in range(1, 9):
        low = (nb[k] >= 0) & (nb[k] < idx)
        want[k, low] = f[k, low] * f[0, nb[k, low]]
    full = oracle.Problem(2, n, 9, d, (1, 1))
    full.ilu0_factor(oracle.DECOMPOSED_FULL)
    assert np.array_equal(full.ilu0_export(), want)
    r = W.uniform_rhs(n[0] * n[1], 5)
    assert np.max(np.abs(full.ilu0_apply(r) - nat.ilu0_apply(r))) <= 1e-13 * np.max(np.abs(nat.ilu0_apply(r)))


@pytest.mark.parametrize("n,sub", [((13, 11), (3, 2)), ((10, 12), (2, 3)), ((7, 9), (7, 1))])
def test_every_block_is_exact_on_its_pattern(n, sub):
    d = _rand9(n, 17 + sub[0])
    pb = oracle.Problem(2, n, 9, d, sub)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    F = pb.ilu0_export()
    nb = neighbours(full_n(n), 9)
    A = assemble(full_n(n), 9, d).toarray()
    for cells in _blocks(pb, n, sub).values():
        L, U = _block_lu(F, nb, cells)
        Ab = A[np.ix_(cells, cells)]
        pat = Ab != 0
        LU = L @ U
        assert np.max(np.abs((LU - Ab)[pat])) <= 1e-12 * np.max(np.abs(Ab))
        # L and U live on the block's pattern
        assert np.all((L - np.eye(len(cells)))[~pat] == 0) and np.all(U[~pat] == 0)


@pytest.mark.parametrize("n,sub", [((9, 8), (2, 2)), ((11, 7), (3, 2))])
def test_five_point_in_nine_point_storage_gives_decomposed_ilu1(n, sub):
    d5 = _rand5(n, 40 + n[0])
    pb = oracle.Problem(2, n, 9, W.embed5in9(d5), sub)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    F = pb.ilu0_export()
    nb = neighbours(full_n(n), 9)
    A = assemble(full_n(n), 5, d5).toarray()
    for cells in _blocks(pb, n, sub).values():
        L, U = _block_lu(F, nb, cells)
        L1, U1, _ = _iluk_dense(A[np.ix_(cells, cells)], 1)
        scale = np.abs(A).max()
        assert np.abs(L - L1).max() <= 1e-12 and np.abs(U - U1).max() <= 1e-12 * scale


def test_five_point_full_factor_is_the_decomposed_ilu0():
    n, sub = (14, 12), (3, 2)
    d = W.diffusion2d(W.smoothed_lognormal_alpha(*n, 8))
    r = W.uniform_rhs(n[0] * n[1], 9)
    a = oracle.Problem(2, n, 5, d, sub)
    a.ilu0_factor(oracle.DECOMPOSED)
    b = oracle.Problem(2, n, 5, d, sub)
    b.ilu0_factor(oracle.DECOMPOSED_FULL)
    za, zb = a.ilu0_apply(r), b.ilu0_apply(r)
    assert np.max(np.abs(za - zb)) <= 1e-13 * np.max(np.abs(za))


@pytest.mark.parametrize("n,sub", [((12, 10), (3, 2)), ((9, 9), (1, 1)), ((16, 6), (4, 2))])
def test_apply_inverts_the_assembled_factor(n, sub):
    """M = (D + L') D^-1 (D + U'): L' the factor's entries on the forward
    phase's implicit sets (within subdomains and the mutual face pairs), U' on
    those of the reverse phase."""
    d = _rand9(n, 61 + n[1])
    pb = oracle.Problem(2, n, 9, d, sub)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    F = pb.ilu0_export()
    tf = pb.fwd_phase()
    jf, _, _, _ = pb.plan_info(oracle.DECOMPOSED, tf)
    jr, _, _, _ = pb.plan_info(oracle.DECOMPOSED, tf ^ 1)
    fn = full_n(n)
    Lp = assemble(fn, 9, F, jmask_bool(jf, 9), include_diag=False).toarray()
    Up = assemble(fn, 9, F, jmask_bool(jr, 9), include_diag=False).toarray()
    D = np.diag(F[0])
    M = (D + Lp) @ np.diag(1.0 / F[0]) @ (D + Up)
    r = W.uniform_rhs(n[0] * n[1], 62)
    z = pb.ilu0_apply(r)
    assert np.max(np.abs(M @ z - r)) <= 1e-12 * np.max(np.abs(r))


def test_full_factor_needs_fewer_iterations_than_dilu():
    n, sub = 48, (3, 3)
    d = W.convdiff9(n, 6.0, 1.1)
    b = W.uniform_rhs(n * n, 12)
    counts = {}
    for mode in (oracle.DECOMPOSED, oracle.DECOMPOSED_FULL):
        pb = oracle.Problem(2, (n, n), 9, d, sub)
        pb.ilu0_factor(mode)
        _, info = pb.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.DECOMPOSED, 1.0, 1e-8, 2000, b)
        assert info["status"] == 0
        counts[mode] = info["iters"]
    assert counts[oracle.DECOMPOSED_FULL] < counts[oracle.DECOMPOSED]
