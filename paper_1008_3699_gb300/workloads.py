"""Seeded synthetic inputs: structured n-diagonal matrices and right-hand sides.

This module only builds inputs. It holds none of the sweep, factorisation or
Krylov arithmetic, and it is the one module that both the CUDA path (tests,
bench) and the CPU oracle receive their inputs from.

Matrices are returned diagonal-major, shape (s, N), cells numbered naturally
with x fastest, entry k of row i being A(i, i + off_k) in the stencil order

    3-pt (1D): C W E
    5-pt (2D): C W E S N
    7-pt (3D): C W E S N B F
    9-pt (2D): C W E S N SW SE NW NE

Entries that would point outside the grid are stored as 0 (homogeneous
Dirichlet values folded into the right-hand side). Discretisations follow
Eq. (d1d)/(d2d) of the paper: second-order finite differences, face
coefficients by harmonic averaging of the cell coefficients, every equation
multiplied through by h^2 so that A is scale-free.

All random draws use numpy's counter-based Philox generator.
"""
from __future__ import annotations

import math

import numpy as np

STENCIL_OFFSETS = {
    3: ((0, 0, 0), (-1, 0, 0), (1, 0, 0)),
    5: ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)),
    7: ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)),
    9: ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
        (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0)),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform_rhs(n_cells: int, seed: int) -> np.ndarray:
    """b ~ U[-1, 1], i.i.d., fp64."""
    return rng(seed).uniform(-1.0, 1.0, size=n_cells)


def _zero_outside(diags: np.ndarray, shape: tuple[int, ...], stencil: int) -> np.ndarray:
    """Zero every entry whose neighbour lies outside the grid."""
    nz = shape[2] if len(shape) > 2 else 1
    ny = shape[1] if len(shape) > 1 else 1
    nx = shape[0]
    view = diags.reshape(stencil, nz, ny, nx)
    for k, (ox, oy, oz) in enumerate(STENCIL_OFFSETS[stencil]):
        if ox < 0:
            view[k, :, :, 0] = 0.0
        if ox > 0:
            view[k, :, :, nx - 1] = 0.0
        if oy < 0:
            view[k, :, 0, :] = 0.0
        if oy > 0:
            view[k, :, ny - 1, :] = 0.0
        if oz < 0:
            view[k, 0, :, :] = 0.0
        if oz > 0:
            view[k, nz - 1, :, :] = 0.0
    return diags


def laplace1d(n: int) -> tuple[np.ndarray, np.ndarray]:
    """1D model of the numerical section: -u'' = 0 on n interior points of a
    uniform grid with u(0) = 0, u(1) = 1 (exact solution u = x). Returns
    (diags (3, n), b) with b carrying the Dirichlet value of the right end."""
    d = np.zeros((3, n))
    d[0] = 2.0
    d[1] = -1.0
    d[2] = -1.0
    d[1, 0] = 0.0
    d[2, n - 1] = 0.0
    b = np.zeros(n)
    b[n - 1] = 1.0
    return d, b


def poisson2d(nx: int, ny: int) -> np.ndarray:
    """5-point Laplacian [4, -1, -1, -1, -1], homogeneous Dirichlet."""
    d = np.empty((5, nx * ny))
    d[0] = 4.0
    d[1:] = -1.0
    return _zero_outside(d, (nx, ny), 5)


def poisson3d(nx: int, ny: int, nz: int) -> np.ndarray:
    """7-point Laplacian [6, -1 x 6], homogeneous Dirichlet."""
    d = np.empty((7, nx * ny * nz))
    d[0] = 6.0
    d[1:] = -1.0
    return _zero_outside(d, (nx, ny, nz), 7)


def box_filter(a: np.ndarray, width: int = 5) -> np.ndarray:
    """Mean over the width x width window, truncated at the domain edge
    (each cell averages the in-range cells of its window only)."""
    r = width // 2
    ny, nx = a.shape
    c = np.zeros((ny + 1, nx + 1))
    c[1:, 1:] = np.cumsum(np.cumsum(a, axis=0), axis=1)
    y0 = np.clip(np.arange(ny) - r, 0, ny)
    y1 = np.clip(np.arange(ny) + r + 1, 0, ny)
    x0 = np.clip(np.arange(nx) - r, 0, nx)
    x1 = np.clip(np.arange(nx) + r + 1, 0, nx)
    s = (c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0])
    cnt = (y1 - y0)[:, None] * (x1 - x0)[None, :]
    return s / cnt


def diffusion2d(alpha: np.ndarray) -> np.ndarray:
    """5-point discretisation of -div(alpha grad u) (Eq. d2d with beta = 0) on a
    uniform grid, alpha given per cell as an (ny, nx) array. Face values are
    harmonic means of the two cells; a boundary face (towards the Dirichlet
    value) uses the cell's own alpha. Multiplied through by h^2."""
    ny, nx = alpha.shape
    hm = lambda p, q: 2.0 * p * q / (p + q)
    aE = np.empty_like(alpha)
    aW = np.empty_like(alpha)
    aN = np.empty_like(alpha)
    aS = np.empty_like(alpha)
    aE[:, :-1] = hm(alpha[:, :-1], alpha[:, 1:])
    aE[:, -1] = alpha[:, -1]
    aW[:, 1:] = aE[:, :-1]
    aW[:, 0] = alpha[:, 0]
    aN[:-1, :] = hm(alpha[:-1, :], alpha[1:, :])
    aN[-1, :] = alpha[-1, :]
    aS[1:, :] = aN[:-1, :]
    aS[0, :] = alpha[0, :]
    d = np.empty((5, nx * ny))
    d[0] = (aE + aW + aN + aS).ravel()
    d[1] = -aW.ravel()
    d[2] = -aE.ravel()
    d[3] = -aS.ravel()
    d[4] = -aN.ravel()
    return _zero_outside(d, (nx, ny), 5)


def smoothed_lognormal_alpha(nx: int, ny: int, seed: int) -> np.ndarray:
    """alpha = box5x5(exp(N(0, 1))) per cell."""
    g = rng(seed)
    return box_filter(np.exp(g.standard_normal((ny, nx))), 5)


def loguniform_alpha(nx: int, ny: int, seed: int, lo: float = 1.0, hi: float = 100.0) -> np.ndarray:
    g = rng(seed)
    return np.exp(g.uniform(math.log(lo), math.log(hi), size=(ny, nx)))


def convdiff9(n: int, peclet: float, theta: float) -> np.ndarray:
    """9-point convection-diffusion -lap(u) + Pe (cos t, sin t) . grad(u) on an
    n x n interior grid, h = 1/(n+1): Laplacian (1/(6h^2)) [-1 -4 -1; -4 20 -4;
    -1 -4 -1], central differences of the convection term on the face
    neighbours. Multiplied through by h^2 (nonsymmetric for Pe > 0)."""
    h = 1.0 / (n + 1)
    vx = peclet * math.cos(theta) * h / 2.0
    vy = peclet * math.sin(theta) * h / 2.0
    d = np.empty((9, n * n))
    d[0] = 20.0 / 6.0
    d[1] = -4.0 / 6.0 - vx   # W
    d[2] = -4.0 / 6.0 + vx   # E
    d[3] = -4.0 / 6.0 - vy   # S
    d[4] = -4.0 / 6.0 + vy   # N
    d[5:] = -1.0 / 6.0
    return _zero_outside(d, (n, n), 9)


# ---------------------------------------------------------------------------
# The five workloads (seed = 1000 + workload number).
# ---------------------------------------------------------------------------

def poisson64_problem():
    """64 x 64 Poisson, 2 x 2 subdomains, omega = 2/(1+sin(pi/65))."""
    n = 64
    return dict(dim=2, n=(n, n, 1), stencil=5, diags=poisson2d(n, n), b=uniform_rhs(n * n, 1001),
                sub=(2, 2, 1), omega=2.0 / (1.0 + math.sin(math.pi / (n + 1))))


def varcoef2d_problem(n: int = 2048, sub: int = 16, seed: int = 1002):
    """n x n variable-coefficient diffusion, alpha = box5x5(exp(N(0,1)))."""
    alpha = smoothed_lognormal_alpha(n, n, seed)
    return dict(dim=2, n=(n, n, 1), stencil=5, diags=diffusion2d(alpha),
                b=uniform_rhs(n * n, seed + 100), sub=(sub, sub, 1))


def poisson3d_problem(n: int = 256, sub: int = 8, seed: int = 1003):
    return dict(dim=3, n=(n, n, n), stencil=7, diags=poisson3d(n, n, n),
                b=uniform_rhs(n ** 3, seed), sub=(sub, sub, sub))


def embed5in9(diags5: np.ndarray) -> np.ndarray:
    """The same matrix in 9-point storage (C W E S N SW SE NW NE), the four
    diagonal entries zero."""
    d = np.zeros((9, diags5.shape[1]))
    d[:5] = diags5
    return d


def eikonal_problem(n: int = 2048, sub: int = 16, seed: int = 1006, sources: int = 4):
    """Travel times on an n x n grid of the unit square (h = 1/n) through a
    heterogeneous medium: slowness f = box5x5(exp(N(0, 1))) per cell, `sources`
    point sources at seeded random cells (u = 0 there, +inf elsewhere)."""
    g = rng(seed)
    f = box_filter(np.exp(g.standard_normal((n, n))), 5).ravel()
    src = np.unique(g.integers(0, n * n, size=sources))
    u0 = np.full(n * n, np.inf)
    u0[src] = 0.0
    return dict(n=(n, n), h=1.0 / n, f=f, u0=u0, sources=src, sub=(sub, sub))


def batched_problems(count: int = 512, lo: int = 32, hi: int = 512, seed: int = 1004):
    """count independent variable-coefficient 5-point problems, sides uniform
    in [lo, hi] independently, alpha log-uniform in [1, 100] per cell."""
    g = rng(seed)
    sides = g.integers(lo, hi + 1, size=(count, 2))
    out = []
    for p in range(count):
        nx, ny = int(sides[p, 0]), int(sides[p, 1])
        alpha = loguniform_alpha(nx, ny, seed * 1000 + 2 * p)
        out.append(dict(dim=2, n=(nx, ny, 1), stencil=5, diags=diffusion2d(alpha),
                        b=uniform_rhs(nx * ny, seed * 1000 + 2 * p + 1)))
    return out


def serving_trace(count: int, rate: float = 2000.0, seed: int = 1005,
                  side2d=(64, 2048), side3d=(32, 192)):
    """Poisson-arrival request trace: half 2D 9-point convection-diffusion
    (Pe ~ U[0,10], theta ~ U[0, 2 pi)), half 3D 7-point Poisson; sides
    log-uniform in the given ranges. Returns (arrival_times, request specs);
    matrices are built lazily by build_request()."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    reqs = []
    for k in range(count):
        if g.uniform() < 0.5:
            side = int(round(math.exp(g.uniform(math.log(side2d[0]), math.log(side2d[1])))))
            reqs.append(dict(kind="convdiff9", side=side, peclet=float(g.uniform(0, 10)),
                             theta=float(g.uniform(0, 2 * math.pi)), seed=seed * 100000 + k))
        else:
            side = int(round(math.exp(g.uniform(math.log(side3d[0]), math.log(side3d[1])))))
            reqs.append(dict(kind="poisson3d", side=side, seed=seed * 100000 + k))
    return t, reqs


def build_request(spec: dict) -> dict:
    if spec["kind"] == "convdiff9":
        n = spec["side"]
        return dict(dim=2, n=(n, n, 1), stencil=9, diags=convdiff9(n, spec["peclet"], spec["theta"]),
                    b=uniform_rhs(n * n, spec["seed"]))
    n = spec["side"]
    return dict(dim=3, n=(n, n, n), stencil=7, diags=poisson3d(n, n, n),
                b=uniform_rhs(n ** 3, spec["seed"]))
