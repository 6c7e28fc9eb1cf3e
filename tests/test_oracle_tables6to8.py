"""Pin the oracle's 2D sweeps to Tables 6-8 of the paper (2D Laplace model
problem, 51^2, 101^2 and 151^2 grids, omega = 1, 1.25, 1.5).

Reading of the tables used here (the text does not state it): the printed
L1 error is one third of the mean absolute error over all grid points, the
boundary points included. Equivalently, the iteration stops once that mean is
below 3e-3. Under this reading, every printed iteration count of the natural
row-wise (R) and frontal (F) rows is reproduced exactly, and their printed L1
errors to within the printing precision on 51^2 (to 5e-5 relative on the
finer grids). With the plain mean, the natural counts come out 27 % higher at
every grid and omega. The rest follows Table 1's reading: "N x N" counts grid
points including the boundary, one sweep is one iteration, and u0 = 0.

- R: natural lexicographic SOR starting at the SW corner;
- F: one subdomain, alternating the first two phases of the 2D schedule (start
  corners NE, then SW);
- P(px x py): the decomposed sweep converges at least as fast as the printed
  count on every topology, and never faster than the frontal sweep by more
  than a few iterations. The oracle couples every face pair whose subdomains
  both start at the interface, as the printed systems do. The paper's own
  code needed 0.2-40 % more sweeps than its frontal sweep.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tables6to8_2d.txt")
GRIDS = (51, 101, 151)
NE, SW = 3, 0


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        om, name = float(f[0]), f[1]
        rows[(om, name)] = {g: (int(f[2 + 2 * k]), float(f[3 + 2 * k])) for k, g in enumerate(GRIDS)}
    return rows


TABLE = _table()


def _model(npts):
    """Interior unknowns of the 5-point Laplacian on npts x npts points, u = x y
    on the boundary (nonzero on x = 1 and y = 1 only)."""
    n = npts - 2
    h = 1.0 / (npts - 1)
    s = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(s, s, indexing="xy")
    b = np.zeros((n, n))
    b[:, -1] += s  # neighbour on x = 1 carries u = y (rows are y)
    b[-1, :] += s  # neighbour on y = 1 carries u = x
    return W.poisson2d(n, n), b.ravel(), (X * Y).ravel(), n


def _iterate(orc, npts, sub, omega, mode, phase_of, library=None):
    d, b, exact, n = _model(npts)
    pb = orc.Problem(2, (n, n), 5, d, sub, library=library)
    x = np.zeros(n * n)
    k = 0
    while True:
        x = pb.sor_sweep(mode, phase_of(k), omega, b, x)
        k += 1
        l1 = np.abs(x - exact).sum() / (npts * npts) / 3.0
        if l1 < 1e-3:
            return k, l1
        assert k < 20000


CELLS = [(om, g) for om in (1.0, 1.25, 1.5) for g in (51, 101)] + [(1.5, 151)]


def _check(got, want, npts):
    assert got[0] == want[0]
    assert abs(got[1] - want[1]) <= (2e-9 if npts == 51 else 1e-7)


@pytest.mark.parametrize("omega,npts", CELLS)
def test_natural_row_order_matches_tables6to8(orc, omega, npts):
    got = _iterate(orc, npts, (1, 1), omega, orc.NATURAL, lambda k: 0)
    _check(got, TABLE[(omega, "R")][npts], npts)


@pytest.mark.parametrize("omega,npts", CELLS)
def test_frontal_sweeping_alternates_ne_and_sw(orc, omega, npts):
    assert [orc.base_corner(2, t) for t in (0, 1)] == [NE, SW]
    got = _iterate(orc, npts, (1, 1), omega, orc.DECOMPOSED, lambda k: k & 1)
    _check(got, TABLE[(omega, "F")][npts], npts)


@pytest.mark.parametrize("omega", [1.0, 1.25, 1.5])
def test_decomposed_sweep_is_at_least_as_fast_as_printed(orc, omega):
    frontal = TABLE[(omega, "F")][51][0]
    for (om, name), row in TABLE.items():
        if om != omega or not name.startswith("P("):
            continue
        px, py = (int(v) for v in name[2:-1].split("x"))
        it, _ = _iterate(orc, 51, (px, py), omega, orc.DECOMPOSED, lambda k: k)
        assert frontal - 5 <= it <= row[51][0], (name, it)


def decomposed_within_table6(library):
    """P(5x5) at 51^2, omega = 1: between the frontal count and the printed one."""
    it, _ = _iterate(oracle, 51, (5, 5), 1.0, oracle.DECOMPOSED, lambda k: k, library)
    return TABLE[(1.0, "F")][51][0] - 5 <= it <= TABLE[(1.0, "P(5x5)")][51][0]
