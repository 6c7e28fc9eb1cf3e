"""The oracle's decomposed 2D 5-point sweep against the procedure of Sec. 3,
written out step by step in plain Python (no implicit sets, no dependency
graph):

1. the start corners: subdomains whose start corners meet at one grid vertex
   solve their corner cells together (Eq. 2d:sor4b4; two cells where the
   vertex lies on the domain boundary, one cell at a domain corner);
2. the start edges: along an interface at which both subdomains start, the
   cells facing each other are solved in pairs (Eq. 2d:sor2b2), moving away
   from the corner, each pair using the new values of the pair before it; a
   start edge on the domain boundary is updated cell by cell in the same
   order;
3. the interior: the remaining cells in row order of the frame reflected
   along the axes the subdomain sweeps backwards, with the new values of the
   cells before them in the subdomain.

Every value not named as new is the old one (the halo of Sec. 3 "Data
structure"). The schedule: subdomain (0,0) starts at its NE, SW, NW, SE corner
at t = 0..3, and a neighbour along an axis starts at the other end of it
(Sec. 3, "Sweeping directions"). The relaxation factor of a cell is that of
its subdomain's start corner.

The only step the two share is the small dense solve of a coupled system.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

OFF = {1: (-1, 0), 2: (1, 0), 3: (0, -1), 4: (0, 1)}  # W E S N
BASE = [3, 0, 2, 1]  # start corner of subdomain (0,0) at t = 0..3 (bit 0: max x, bit 1: max y)


def _split(n, p):
    q, r = divmod(n, p)
    lo = [k * q + min(k, r) for k in range(p + 1)]
    return [(lo[k], lo[k + 1]) for k in range(p)]


def subdomains(n, sub, t, omega=(1.0, 1.0, 1.0, 1.0)):
    """Bounds, start corner and relaxation factor of every subdomain at phase t."""
    subs = []
    for iy, (y0, y1) in enumerate(_split(n[1], sub[1])):
        for ix, (x0, x1) in enumerate(_split(n[0], sub[0])):
            cs = BASE[t % 4] ^ (ix & 1) ^ ((iy & 1) << 1)
            subs.append(dict(x0=x0, x1=x1, y0=y0, y1=y1, cs=cs, w=omega[cs]))
    return subs


def frame(s, xr, yr):
    """Global cell of reflected coordinates (xr, yr) in subdomain s."""
    x = s["x1"] - 1 - xr if s["cs"] & 1 else s["x0"] + xr
    y = s["y1"] - 1 - yr if s["cs"] & 2 else s["y0"] + yr
    return x, y


def corner_groups(subs):
    """Start-corner cells grouped by the grid vertex (in half-cell units) they
    meet at."""
    groups = {}
    for s in subs:
        x, y = frame(s, 0, 0)
        vx = 2 * x + (1 if s["cs"] & 1 else -1)
        vy = 2 * y + (1 if s["cs"] & 2 else -1)
        groups.setdefault((vx, vy), []).append((x, y))
    return [sorted(c) for c in groups.values()]


def procedural_sweep(n, sub, d, omega, t, b, u):
    nx, ny = n
    A = d.reshape(5, ny, nx)
    uo = u.reshape(ny, nx)
    bb = b.reshape(ny, nx)
    new = {}

    def nb(x, y, k):
        ox, oy = OFF[k]
        xx, yy = x + ox, y + oy
        return (xx, yy) if 0 <= xx < nx and 0 <= yy < ny else None

    subs = subdomains(n, sub, t, omega)
    owner = {}
    for s in subs:
        for y in range(s["y0"], s["y1"]):
            for x in range(s["x0"], s["x1"]):
                owner[(x, y)] = s

    def solve(cells):
        """Relaxed update of a group of cells solved together: the group's
        members, and the cells of a member's own subdomain already in `new`,
        are new; every other value is old (other subdomains sweep at the same
        time)."""
        idx = {c: i for i, c in enumerate(cells)}
        m = len(cells)
        M = np.zeros((m, m))
        r = np.zeros(m)
        for i, (x, y) in enumerate(cells):
            w = owner[(x, y)]["w"]
            aii = A[0, y, x]
            M[i, i] = aii
            r[i] = (1 - w) * aii * uo[y, x] + w * bb[y, x]
            for k in range(1, 5):
                q = nb(x, y, k)
                if q is None:
                    continue
                a = A[k, y, x]
                if q in idx:
                    M[i, idx[q]] += w * a
                else:
                    own = owner[q] is owner[(x, y)] and q in new
                    r[i] -= w * a * (new[q] if own else uo[q[1], q[0]])
        v = np.linalg.solve(M, r) if m > 1 else r / M[0, 0]
        for c, val in zip(cells, v):
            new[c] = val

    def starts_at(s, q):
        """Does subdomain s start on the side facing cell q (in another one)?"""
        x0, y0 = frame(s, 0, 0)
        return (q[0] == x0 + (1 if s["cs"] & 1 else -1) and s["y0"] <= q[1] < s["y1"]) or \
               (q[1] == y0 + (1 if s["cs"] & 2 else -1) and s["x0"] <= q[0] < s["x1"])

    # 1. start corners, grouped by the grid vertex they meet at
    for cells in corner_groups(subs):
        solve(cells)
    # 2. start edges: along x (the start row) and along y (the start column)
    done = set(new)
    for s in subs:
        w_, h_ = s["x1"] - s["x0"], s["y1"] - s["y0"]
        for along, length in ((0, w_), (1, h_)):
            for dist in range(1, length):
                c = frame(s, dist, 0) if along == 0 else frame(s, 0, dist)
                if c in done:
                    continue
                # the neighbour across this start edge, if it also starts there
                k = (4 if s["cs"] & 2 else 3) if along == 0 else (2 if s["cs"] & 1 else 1)
                q = nb(c[0], c[1], k)
                if q is not None and owner[q] is not s and starts_at(owner[q], c):
                    pair = sorted([c, q])
                    solve(pair)
                    done.update(pair)
                else:
                    solve([c])
                    done.add(c)
    # 3. the interior, row by row in the reflected frame
    for s in subs:
        for yr in range(1, s["y1"] - s["y0"]):
            for xr in range(1, s["x1"] - s["x0"]):
                c = frame(s, xr, yr)
                solve([c])
    out = np.empty(nx * ny)
    for (x, y), v in new.items():
        out[x + nx * y] = v
    assert len(new) == nx * ny
    return out


PARTS = [((20, 17), (3, 2)), ((13, 11), (2, 2)), ((9, 12), (9, 4)), ((16, 5), (4, 5)), ((7, 7), (1, 1)),
         ((24, 10), (5, 1)), ((11, 19), (1, 4))]


def _rand5(n, seed):
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.2, 1.0, size=(5, N))
    d = W._zero_outside(d, n, 5)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def procedure_holds(n, sub, library=None):
    """Every phase of the oracle's sweep equals the procedure, to 1e-13."""
    g = np.random.default_rng(5)
    N = n[0] * n[1]
    d = _rand5(n, 6)
    pb = oracle.Problem(2, n, 5, d, sub, library=library)
    omega = g.uniform(0.6, 1.8, size=4)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    for t in range(4):
        got = pb.sor_sweep(oracle.DECOMPOSED, t, omega, b, u)
        want = procedural_sweep(n, sub, d, omega, t, b, u)
        if np.max(np.abs(got - want)) > 1e-13 * np.max(np.abs(want)):
            return False
    return True


@pytest.mark.parametrize("n,sub", PARTS)
def test_sweep_follows_the_procedure_of_sec3(orc, n, sub):
    assert [orc.base_corner(2, t) for t in range(4)] == BASE
    assert procedure_holds(n, sub)


def test_corner_groups_have_the_printed_sizes():
    # 2 x 2 subdomains: at t = 0 all four start at the centre vertex (the 4x4
    # system of Eq. 2d:sor4b4); at t = 1 each starts at a domain corner alone.
    assert sorted(len(g) for g in corner_groups(subdomains((12, 12), (2, 2), 0))) == [4]
    assert sorted(len(g) for g in corner_groups(subdomains((12, 12), (2, 2), 1))) == [1, 1, 1, 1]
    # 3 x 3 at t = 0: one interior vertex with four start corners, two vertices
    # on the domain boundary with two (2x2 systems), one domain corner alone.
    assert sorted(len(g) for g in corner_groups(subdomains((12, 12), (3, 3), 0))) == [1, 2, 2, 4]
    # neighbours along an axis start at opposite ends of it (Sec. 3)
    for t in range(4):
        subs = subdomains((12, 12), (3, 3), t)
        for iy, ix in itertools.product(range(3), range(2)):
            assert subs[iy * 3 + ix]["cs"] ^ subs[iy * 3 + ix + 1]["cs"] == 1
        for iy, ix in itertools.product(range(2), range(3)):
            assert subs[iy * 3 + ix]["cs"] ^ subs[(iy + 1) * 3 + ix]["cs"] == 2
