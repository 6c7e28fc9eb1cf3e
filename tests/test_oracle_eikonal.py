"""Pins of the oracle's fast sweeping (decomposed Gauss-Seidel passes with
Zhao's Godunov update) against facts fixed outside it:

- a hand-worked 1D example (8 cells, 2 subdomains, source at x = 0): the
  values after each of the first four sweeps follow from the sweep schedule
  (which way each subdomain runs at each phase) and from old values across
  the interface;
- the Godunov scheme's closed forms on a uniform medium: values along the
  grid lines through a point source are exact multiples of h, and the
  diagonal neighbour of a source is h (1 + 1/sqrt(2));
- Zhao's theorem (Math. Comp. 74, 2005): for one point source in a uniform
  medium, one pass of each of the four orderings gives the converged
  solution;
- first-order convergence to the exact solution: the distance function
  (f = 1) and u = r^2 (f = 2 r), error falling with h;
- the fixed point does not depend on the partition (the discrete Godunov
  system has one solution);
- planted mistakes in a copy of the oracle each fail one of these.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle

INF = np.inf


def _grid_xy(nx, ny):
    i = np.arange(nx * ny)
    return i % nx, i // nx


def pin_worked_1d(L):
    E = oracle.Eikonal((8, 1), 1.0, np.ones(8), (2, 1), library=L)
    u = oracle.eikonal_init(8, [0])
    want = [
        [0, 1, INF, INF, INF, INF, INF, INF],  # t=0: left part right-to-left, right part left-to-right
        [0, 1, 2, 3, INF, INF, INF, INF],      # t=1: left part left-to-right; right part sees old inf
        [0, 1, 2, 3, 4, INF, INF, INF],        # t=2: right part right-to-left, reaches x=4 last
        [0, 1, 2, 3, 4, 5, 6, 7],              # t=3: right part left-to-right
    ]
    for t in range(4):
        u, _ = E.sweep(t, u)
        if not np.array_equal(u, np.array(want[t], dtype=float)):
            return False
    return True


def pin_axis_and_diagonal(L):
    n, h = 33, 1.0 / 64
    E = oracle.Eikonal((n, n), h, np.ones(n * n), (1, 1), library=L)
    s = 16 * n + 16
    u, info = E.solve(oracle.eikonal_init(n * n, [s]))
    k = np.abs(np.arange(n) - 16) * h
    row, col = u[16 * n:17 * n], u[16::n]
    diag = u[s + n + 1]
    return (info["converged"] and np.array_equal(row, k) and np.array_equal(col, k)
            and abs(diag - h * (1 + 1 / np.sqrt(2))) <= 1e-16)


def pin_zhao_four_sweeps(L):
    nx, ny, h = 40, 29, 0.05
    E = oracle.Eikonal((nx, ny), h, np.ones(nx * ny), (1, 1), library=L)
    u = oracle.eikonal_init(nx * ny, [11 * nx + 27])
    for t in range(4):
        u, _ = E.sweep(t, u)
    u8, info = E.solve(u)
    return info["sweeps"] == 4 and np.array_equal(u8, u) and np.isfinite(u).all()


def _error(n, case, L):
    h = 2.0 / (n - 1)  # [-1, 1]^2, source at the centre cell
    x, y = _grid_xy(n, n)
    X, Y = (x - (n - 1) // 2) * h, (y - (n - 1) // 2) * h
    r = np.hypot(X, Y)
    f, exact = (np.ones(n * n), r) if case == "dist" else (2 * r, r * r)
    E = oracle.Eikonal((n, n), h, f, (1, 1), library=L)
    u, info = E.solve(oracle.eikonal_init(n * n, [(n - 1) // 2 * n + (n - 1) // 2]))
    return np.abs(u - exact).max() if info["converged"] else np.inf


def pin_convergence(L):
    for case, c in (("dist", 0.6), ("r2", 3.0)):
        e = [_error(n, case, L) for n in (33, 65, 129)]
        h = [2.0 / 32, 2.0 / 64, 2.0 / 128]
        if not (e[0] > e[1] > e[2]):
            return False
        # first order up to the logarithm of the point source
        if any(ek > c * hk * max(1.0, np.log(1 / hk)) for ek, hk in zip(e, h)):
            return False
    return True


def _speed(nx, ny, seed):
    g = np.random.default_rng(seed)
    return np.exp(0.5 * g.standard_normal(nx * ny))


def pin_partition_free(L):
    nx, ny, h = 37, 30, 0.1
    f = _speed(nx, ny, 9)
    u0 = oracle.eikonal_init(nx * ny, [3 * nx + 5, 25 * nx + 30])
    ref, i1 = oracle.Eikonal((nx, ny), h, f, (1, 1), library=L).solve(u0)
    for sub in ((2, 2), (3, 2), (5, 4)):
        u, info = oracle.Eikonal((nx, ny), h, f, sub, library=L).solve(u0)
        if not info["converged"] or np.abs(u - ref).max() > 1e-12 * np.abs(ref).max():
            return False
    return i1["converged"]


PINS = [pin_worked_1d, pin_axis_and_diagonal, pin_zhao_four_sweeps, pin_convergence, pin_partition_free]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin_holds(pin):
    assert pin(oracle.lib())


def test_decomposed_needs_more_sweeps_than_sequential():
    nx = ny = 96
    f = _speed(nx, ny, 3)
    u0 = oracle.eikonal_init(nx * ny, [40 * nx + 50])
    _, seq = oracle.Eikonal((nx, ny), 1 / 96, f, (1, 1)).solve(u0)
    _, dec = oracle.Eikonal((nx, ny), 1 / 96, f, (4, 4)).solve(u0)
    assert seq["converged"] and dec["converged"]
    assert seq["sweeps"] <= dec["sweeps"] <= 8 * seq["sweeps"]


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.Eikonal((8, 8), 0.0, np.ones(64))
    with pytest.raises(ValueError):
        oracle.Eikonal((8, 8), 1.0, np.ones(64), (9, 1))


# --- planted mistakes ---------------------------------------------------------

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")

MUTANTS = [
    ("  return (a + b + std::sqrt(2.0 * (fh * fh) - d * d)) * 0.5;",
     "  return (a + b - std::sqrt(2.0 * (fh * fh) - d * d)) * 0.5;"),
    ("  return (a + b + std::sqrt(2.0 * (fh * fh) - d * d)) * 0.5;",
     "  return (a + b + std::sqrt((fh * fh) - d * d)) * 0.5;"),
    ("  if (!(std::fabs(d) < fh)) return std::min(a, b) + fh;",
     "  if (!(std::fabs(d) < 2.0 * fh)) return std::min(a, b) + fh;"),
    ("  if (!(std::fabs(d) < fh)) return std::min(a, b) + fh;",
     "  if (!(std::fabs(d) < fh)) return std::max(a, b) + fh;"),
    ("        return mine ? un[y * nx + x] : uo[y * nx + x];", "        return un[y * nx + x];"),
    ("        return mine ? un[y * nx + x] : uo[y * nx + x];", "        return uo[y * nx + x];"),
    ("      const int c = subdomain_corner(2, t, idx);", "      const int c = base_corner(2, t);"),
    ("        const int64_t y = (c & 2) ? y1 - 1 - yy : y0 + yy;",
     "        const int64_t y = (c & 1) ? y1 - 1 - yy : y0 + yy;"),
    ("          const double b = std::min(val(x, y - 1), val(x, y + 1));",
     "          const double b = std::min(val(x, y - 1), val(x + 1, y + 1));"),
]


@pytest.mark.parametrize("anchor,replacement", MUTANTS)
def test_pins_catch_planted_mistake(tmp_path, anchor, replacement):
    src = open(SRC).read()
    assert src.count(anchor) == 1, anchor
    path = tmp_path / "mut.cpp"
    path.write_text(src.replace(anchor, replacement))
    out = str(tmp_path / "libmut.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, str(path)],
                   check=True)
    L = oracle.lib(out)
    assert not all(p(L) for p in PINS)
