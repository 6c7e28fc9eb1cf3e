"""The oracle's decomposed 2D 5-point sweep against the procedure of Sec. 3
(and the 3D 7-point sweep against Sec. 4, at the end of the file), written out
step by step in plain Python (no implicit sets, no dependency
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


# ---------------------------------------------------------------------------
# 3D (Sec. 4): the same procedure for the 7-point stencil
# ---------------------------------------------------------------------------

OFF3 = {1: (-1, 0, 0), 2: (1, 0, 0), 3: (0, -1, 0), 4: (0, 1, 0), 5: (0, 0, -1), 6: (0, 0, 1)}


def base_corner_3d(t):
    """Start corner of subdomain (0,0,0) at phase t: within each pair of sweeps
    the direction reverses; pair g starts from the all-ones corner with the
    bits of g flipped on x and y (the 3D schedule, which the paper leaves
    open)."""
    g = (t // 2) % 4
    c = 7 ^ (g & 1) ^ (((g >> 1) & 1) << 1)
    return c ^ 7 if t % 2 else c


def procedural_sweep_3d(n, sub, d, omega, t, b, u):
    """Sec. 4 in the form that needs no case list: every subdomain visits its
    cells in lexicographic (z, y, x) order of its reflected frame; a cell that
    lies on start faces with a neighbouring subdomain behind them is solved
    together with the cells facing it across those faces (all subdomains
    around a start vertex, edge or face start there): 8 cells at an interior
    start vertex (the 8x8 system), 4 along a start edge, 2 across a start
    face, 1 inside. A coupled group is solved once, when its first member is
    reached; a cell's own subdomain supplies new values for the cells it has
    visited, everything else is old."""
    nx, ny, nz = n
    A = d.reshape(7, nz, ny, nx)
    uo = u.reshape(nz, ny, nx)
    bb = b.reshape(nz, ny, nx)
    parts = [_split(n[a], sub[a]) for a in range(3)]
    subs = []
    for iz, (z0, z1) in enumerate(parts[2]):
        for iy, (y0, y1) in enumerate(parts[1]):
            for ix, (x0, x1) in enumerate(parts[0]):
                cs = base_corner_3d(t) ^ (ix & 1) ^ ((iy & 1) << 1) ^ ((iz & 1) << 2)
                subs.append(dict(lo=(x0, y0, z0), hi=(x1, y1, z1), cs=cs, w=omega[cs]))
    owner = {}
    for s in subs:
        for c in itertools.product(*(range(s["lo"][a], s["hi"][a]) for a in range(3))):
            owner[c] = s
    new = {}

    def cell(s, r):
        return tuple(s["hi"][a] - 1 - r[a] if s["cs"] >> a & 1 else s["lo"][a] + r[a] for a in range(3))

    def nb(c, k):
        q = tuple(c[a] + OFF3[k][a] for a in range(3))
        return q if all(0 <= q[a] < n[a] for a in range(3)) else None

    def solve(cells):
        idx = {c: i for i, c in enumerate(cells)}
        m = len(cells)
        M = np.zeros((m, m))
        r = np.zeros(m)
        for i, c in enumerate(cells):
            x, y, z = c
            w = owner[c]["w"]
            M[i, i] = A[0, z, y, x]
            r[i] = (1 - w) * A[0, z, y, x] * uo[z, y, x] + w * bb[z, y, x]
            for k in range(1, 7):
                q = nb(c, k)
                if q is None:
                    continue
                a = A[k, z, y, x]
                if q in idx:
                    M[i, idx[q]] += w * a
                else:
                    own = owner[q] is owner[c] and q in new
                    r[i] -= w * a * (new[q] if own else uo[q[2], q[1], q[0]])
        v = np.linalg.solve(M, r) if m > 1 else r / M[0, 0]
        for c, val in zip(cells, v):
            new[c] = val

    for s in subs:
        ext = [s["hi"][a] - s["lo"][a] for a in range(3)]
        for rz, ry, rx in itertools.product(range(ext[2]), range(ext[1]), range(ext[0])):
            c = cell(s, (rx, ry, rz))
            if c in new:
                continue
            # the start faces this cell lies on that have a subdomain behind them
            steps = []
            for a, ra in enumerate((rx, ry, rz)):
                if ra == 0:
                    q = list(c)
                    q[a] += 1 if s["cs"] >> a & 1 else -1
                    if 0 <= q[a] < n[a]:
                        steps.append((a, q[a] - c[a]))
            group = []
            for m in range(len(steps) + 1):
                for sel in itertools.combinations(steps, m):
                    q = list(c)
                    for a, dlt in sel:
                        q[a] += dlt
                    group.append(tuple(q))
            solve(sorted(group))
    out = np.empty(nx * ny * nz)
    for (x, y, z), v in new.items():
        out[x + nx * (y + ny * z)] = v
    assert len(new) == nx * ny * nz
    return out


PARTS3 = [((6, 5, 7), (2, 2, 3)), ((5, 4, 6), (5, 1, 2)), ((7, 6, 5), (3, 2, 2)), ((4, 4, 4), (1, 1, 1)),
          ((6, 6, 6), (2, 2, 2))]


def _rand7(n, seed):
    g = np.random.default_rng(seed)
    N = int(np.prod(n))
    d = -g.uniform(0.2, 1.0, size=(7, N))
    d = W._zero_outside(d, n, 7)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def procedure3d_holds(n, sub, library=None):
    """Every phase of the oracle's 3D sweep equals the procedure, to 1e-13."""
    g = np.random.default_rng(7)
    N = int(np.prod(n))
    d = _rand7(n, 8)
    pb = oracle.Problem(3, n, 7, d, sub, library=library)
    omega = g.uniform(0.6, 1.8, size=8)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    for t in range(8):
        got = pb.sor_sweep(oracle.DECOMPOSED, t, omega, b, u)
        want = procedural_sweep_3d(n, sub, d, omega, t, b, u)
        if np.max(np.abs(got - want)) > 1e-13 * np.max(np.abs(want)):
            return False
    return True


@pytest.mark.parametrize("n,sub", PARTS3)
def test_3d_sweep_follows_the_procedure_of_sec4(orc, n, sub):
    assert [orc.base_corner(3, t) for t in range(8)] == [base_corner_3d(t) for t in range(8)]
    assert procedure3d_holds(n, sub)


def test_3d_corner_system_is_8x8_with_32_nonzeros():
    # 2 x 2 x 2 subdomains at t = 0 all start at the centre vertex: one group
    # of 8 cells; each cell has 3 coupled neighbours in it, so the system has
    # 8 diagonal + 24 off-diagonal = 32 nonzeros (Sec. 4).
    n = (6, 6, 6)
    cells = []
    for iz, iy, ix in itertools.product(range(2), range(2), range(2)):
        cs = base_corner_3d(0) ^ ix ^ (iy << 1) ^ (iz << 2)
        lo = (3 * ix, 3 * iy, 3 * iz)
        cells.append(tuple(lo[a] + (2 if cs >> a & 1 else 0) for a in range(3)))
    assert len(set(cells)) == 8
    adj = sum(1 for p in cells for q in cells if sum(abs(p[a] - q[a]) for a in range(3)) == 1)
    assert 8 + adj == 32
