"""Property-based pins of the oracle's decomposed sweep (hypothesis, CPU).

Over random grids (sides 1..9, 2D 5-point / 9-point and 3D 7-point), random
Cartesian partitions (one-cell-thick subdomains included), every schedule
phase and random relaxation factors per start corner, one decomposed sweep
solves its splitting equation (D + w L_J) u+ = ((1 - w) D - w U_J) u + w b
(Eq. ca2d:matiter) to 1e-12 against scipy's sparse direct solve, and the
implicit set keeps its defining properties: nothing outside the grid, and
across an interface only face neighbours, only in mutual pairs (the 9-point
diagonal neighbours across an interface stay explicit).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from tests.oracle_dense import assemble, full_n, jmask_bool, neighbours

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


def _part(nv, p):
    """Part index of every coordinate: n cells into p parts, the first n mod p one longer."""
    q, r = divmod(nv, p)
    lens = [q + (1 if k < r else 0) for k in range(p)]
    return np.repeat(np.arange(p), lens)


def _diags(n, stencil, seed):
    g = np.random.default_rng(seed)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(stencil, N))
    d[neighbours(n, stencil) < 0] = 0.0
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


@st.composite
def problems(draw):
    kind = draw(st.sampled_from([(2, 5), (2, 9), (3, 7)]))
    dim, stencil = kind
    n = tuple(draw(st.integers(1, 9 if dim == 2 else 5)) for _ in range(dim))
    sub = tuple(draw(st.integers(1, v)) for v in n)
    seed = draw(st.integers(0, 2 ** 20))
    return dim, stencil, n, sub, seed


@hypothesis.settings(max_examples=40, deadline=None)
@hypothesis.given(problems())
def test_sweep_solves_its_splitting_equation(orc, prob):
    dim, stencil, n, sub, seed = prob
    fn = full_n(n)
    N = int(np.prod(fn))
    d = _diags(fn, stencil, seed)
    g = np.random.default_rng(seed + 1)
    pb = orc.Problem(dim, n, stencil, d, sub)
    omega = g.uniform(0.6, 1.8, size=2 ** dim)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    nb = neighbours(fn, stencil)
    for t in range(2 ** dim):
        x = pb.sor_sweep(orc.DECOMPOSED, t, omega, b, u)
        jm, corner, _, _ = pb.plan_info(orc.DECOMPOSED, t)
        J = jmask_bool(jm, stencil)
        U = ~J & (nb >= 0)
        U[0] = False
        w = omega[corner]
        L = assemble(fn, stencil, d, J, include_diag=False)
        Um = assemble(fn, stencil, d, U, include_diag=False)
        lhs = (sp.diags(d[0]) + sp.diags(w) @ L).tocsc()
        rhs = (sp.diags(1 - w) @ sp.diags(d[0]) - sp.diags(w) @ Um) @ u + w * b
        ref = spla.spsolve(lhs, rhs) if N > 1 else rhs / lhs.toarray()[0, 0]
        assert np.max(np.abs(x - ref)) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300)
        # implicit set: no entry points outside the grid
        assert not np.any(J[1:] & (nb[1:] < 0))
        # across an interface only face neighbours are implicit, and only in mutual pairs
        idx = np.arange(N)
        coords = [idx % fn[0], (idx // fn[0]) % fn[1], idx // (fn[0] * fn[1])]
        parts = [_part(fn[a], (list(sub) + [1, 1])[a])[coords[a]] for a in range(3)]
        sid = parts[0] + 1000 * (parts[1] + 1000 * parts[2])
        opp = {1: 2, 2: 1, 3: 4, 4: 3, 5: 6, 6: 5}
        for k in range(1, stencil):
            has = nb[k] >= 0
            cross = np.zeros(N, dtype=bool)
            cross[has] = sid[has] != sid[nb[k][has]]
            sel = J[k] & cross
            if stencil == 9 and k >= 5:
                assert not np.any(sel), "diagonal neighbour across an interface is implicit"
                continue
            j = nb[k][sel]
            assert np.all(J[opp[k]][j]), "non-mutual implicit pair across an interface"
