"""ILU(1) of a 5-point matrix in natural order, as the 9-point factor.

On a 5-point matrix in natural order, level-of-fill ILU(1) fills exactly the
two diagonal positions (x+1, y-1) and (x-1, y+1); the other two corners of the
9-point molecule never fill. So the natural ILU(0) of the 9-point pattern,
applied to the matrix stored with zero corners, is its ILU(1). The pin is a
textbook level-of-fill ILU(p) (Saad, Iterative Methods for Sparse Linear
Systems, Alg. 10.5), written out densely here on small grids, against the
oracle's 9-point factor.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, neighbours


def _iluk_dense(A, p):
    """Dense IKJ ILU(p) with levels of fill; returns unit-lower L and U."""
    n = A.shape[0]
    a = A.astype(float).copy()
    lev = np.where(a != 0, 0, np.iinfo(np.int64).max // 4)
    for i in range(1, n):
        for k in range(i):
            if lev[i, k] > p or a[i, k] == 0 and lev[i, k] > 0:
                continue
            a[i, k] /= a[k, k]
            for j in range(k + 1, n):
                if a[k, j] == 0 and lev[k, j] > p:
                    continue
                new = lev[i, k] + lev[k, j] + 1
                if new < lev[i, j]:
                    lev[i, j] = new
                a[i, j] -= a[i, k] * a[k, j]
        drop = lev[i] > p
        a[i, drop] = 0.0
    L = np.tril(a, -1) + np.eye(n)
    U = np.triu(a)
    return L, U, lev


def _rand5(n, seed):
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.2, 1.0, size=(5, N))
    d = W._zero_outside(d, (n[0], n[1]), 5)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


@pytest.mark.parametrize("n", [(7, 6), (5, 9), (3, 4)])
def test_ilu1_equals_nine_point_natural_factor(n):
    d5 = _rand5(n, sum(n))
    fn = full_n(n)
    A = assemble(fn, 5, d5).toarray()
    L1, U1, lev = _iluk_dense(A, 1)
    pb = oracle.Problem(2, n, 9, W.embed5in9(d5), (1, 1))
    pb.ilu0_factor(oracle.NATURAL)
    f = pb.ilu0_export()
    nb = neighbours(fn, 9)
    N = nb.shape[1]
    idx = np.arange(N)
    lower, upper = (nb >= 0) & (nb < idx), nb > idx
    L = assemble(fn, 9, f, lower, include_diag=False).toarray() + np.eye(N)
    U = assemble(fn, 9, f, upper, include_diag=True).toarray()
    scale = np.abs(A).max()
    assert np.abs(L - L1).max() <= 1e-12 and np.abs(U - U1).max() <= 1e-12 * scale
    # fill only at (x+1, y-1) and (x-1, y+1): level 1; the other corners stay zero
    assert np.all(f[5] == 0.0) and np.all(f[8] == 0.0)
    assert (lev <= 1).sum() == ((L != 0) | (U != 0)).sum()


def test_ilu1_beats_ilu0_on_the_varcoef_operator():
    n = 64
    d5 = W.diffusion2d(W.smoothed_lognormal_alpha(n, n, 3))
    b = W.uniform_rhs(n * n, 4)
    p0 = oracle.Problem(2, (n, n), 5, d5, (1, 1))
    p0.ilu0_factor(oracle.NATURAL)
    _, i0 = p0.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.NATURAL, 1.0, 1e-8, 2000, b)
    p1 = oracle.Problem(2, (n, n), 9, W.embed5in9(d5), (1, 1))
    p1.ilu0_factor(oracle.NATURAL)
    _, i1 = p1.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.NATURAL, 1.0, 1e-8, 2000, b)
    assert i0["status"] == 0 and i1["status"] == 0
    assert i1["iters"] < i0["iters"]
