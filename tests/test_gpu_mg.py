"""Multigrid V-cycle with the decomposed SSOR smoother (mg_apply, and
krylov_solve with NDIAG_PREC_MG) against the oracle's cycle (oracle/mg.py):
one V-cycle element by element, the hierarchy's levels, PCG iteration counts
within one, the argument checks, and at full size (2048^2, 16 x 16 subdomains)
one V-cycle element by element and the solve's iteration count against the
stored oracle count; the 3D 7-point cycle likewise on 3D grids."""
import json
import os

import numpy as np
import pytest

import oracle
import oracle.mg as M
from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "varcoef2048_mg.json")
VTOL = 1e-10  # one V-cycle: |z - z_oracle| <= VTOL * max |z_oracle|


@pytest.fixture(scope="module")
def nd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_3699_gb300 import build, ndiag
    build.build()
    return ndiag


def _matrix(kind, nx, ny, seed):
    if kind == "poisson":
        return W.poisson2d(nx, ny)
    if kind == "loguniform":
        return W.diffusion2d(W.loguniform_alpha(nx, ny, seed, 1.0, 100.0))
    return W.diffusion2d(W.smoothed_lognormal_alpha(nx, ny, seed))


CASES = [
    (300, 260, (3, 3), 0.9, "varcoef", 41),     # 5 levels, 9 x 8 subdomains on level 1
    (257, 131, (2, 1), 0.85, "loguniform", 42),  # odd sides: one-cell-wide aggregates
    (30, 20, (2, 2), 0.9, "poisson", 43),       # one level: SSOR-Richardson only
    (520, 64, (5, 1), 0.95, "varcoef", 44),     # elongated, 5 x 1 then 16 x 2 subdomains
]


@pytest.mark.parametrize("nx,ny,sub,om,kind,seed", CASES)
def test_vcycle_matches_oracle(nd, nx, ny, sub, om, kind, seed):
    import torch
    d = _matrix(kind, nx, ny, seed)
    r = np.random.default_rng(seed).standard_normal(nx * ny)
    H = M.Hierarchy(nx, ny, d, sub, om)
    want = H.vcycle(r)
    h = nd.NDiag(2, (nx, ny), 5, d, sub, "fp64")
    rd = torch.tensor(r, device="cuda")
    z = torch.empty_like(rd)
    h.mg_apply(om, rd, z)
    z1 = z.cpu().numpy()
    assert h.mg_levels() == len(H.levels)
    h.mg_apply(om, rd, z)  # the kept hierarchy gives the same cycle
    z2 = z.cpu().numpy()
    h.close()
    err = np.abs(z1 - want).max() / np.abs(want).max()
    assert err <= VTOL, err
    np.testing.assert_array_equal(z1, z2)


@pytest.mark.parametrize("nx,ny,sub,om,kind,seed", [CASES[0], CASES[1]])
def test_pcg_mg_matches_oracle_count(nd, nx, ny, sub, om, kind, seed):
    import torch
    d = _matrix(kind, nx, ny, seed)
    b = W.uniform_rhs(nx * ny, seed + 100)
    H = M.Hierarchy(nx, ny, d, sub, om)
    xr, info = M.pcg(H, b, 1e-8, 500)
    assert info["status"] == 0
    h = nd.NDiag(2, (nx, ny), 5, d, sub, "fp64")
    bd = torch.tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    res = h.solve(nd.PCG, nd.PREC_MG, bd, x, rtol=1e-8, maxit=500, omega=om)
    h.close()
    assert res["relres"] <= 1e-8
    assert abs(res["iters"] - info["iters"]) <= 1, (res, info)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)


def test_bicgstab_accepts_the_cycle(nd):
    import torch
    nx, ny = 200, 150
    d = _matrix("varcoef", nx, ny, 45)
    h = nd.NDiag(2, (nx, ny), 5, d, (2, 2), "fp64")
    bd = torch.tensor(W.uniform_rhs(nx * ny, 46), device="cuda")
    x = torch.zeros_like(bd)
    res = h.solve(nd.BICGSTAB, nd.PREC_MG, bd, x, rtol=1e-8, maxit=500, omega=0.9)
    h.close()
    assert res["relres"] <= 1e-8 and res["iters"] < 40


def test_refused_configurations(nd):
    import torch
    nx, ny = 40, 40
    d = W.poisson2d(nx, ny)
    b = torch.ones(nx * ny, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    h32 = nd.NDiag(2, (nx, ny), 5, d, (2, 2), "fp32")
    with pytest.raises(nd.NdiagError):
        h32.solve(nd.PCG, nd.PREC_MG, b, x, omega=0.9)
    with pytest.raises(nd.NdiagError):
        h32.mg_apply(0.9, b.float(), x.float())
    h32.close()
    h = nd.NDiag(2, (nx, ny), 5, d, (2, 2), "fp64")
    with pytest.raises(nd.NdiagError):
        h.solve(nd.PCG, nd.PREC_MG, b, x, omega=0.9, mode=nd.NATURAL)
    with pytest.raises(nd.NdiagError):
        h.mg_apply(2.0, b, x)
    assert h.mg_levels() == 0
    h.close()
    h3 = nd.NDiag(3, (16, 16, 16), 7, W.poisson3d(16, 16, 16), (2, 2, 2), "fp32")
    b3 = torch.ones(16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdiagError):
        h3.solve(nd.PCG, nd.PREC_MG, b3, torch.zeros_like(b3), omega=0.9)
    h3.close()
    h9 = nd.NDiag(2, (20, 20), 9, W.convdiff9(20, 1.0, 0.3), (2, 2), "fp64")
    b9 = torch.ones(400, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdiagError):
        h9.solve(nd.PCG, nd.PREC_MG, b9, torch.zeros_like(b9), omega=0.9)
    h9.close()


def test_full_size_vcycle_and_count(nd):
    import torch
    p = W.varcoef2d_problem()
    n, sub, om = p["n"][0], p["sub"], 0.9
    r = np.random.default_rng(47).standard_normal(n * n)
    H = M.Hierarchy(n, n, p["diags"], sub, om)
    want = H.vcycle(r)
    h = nd.NDiag(2, p["n"], 5, p["diags"], sub, "fp64")
    rd = torch.tensor(r, device="cuda")
    z = torch.empty_like(rd)
    h.mg_apply(om, rd, z)
    err = np.abs(z.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= VTOL, err
    assert h.mg_levels() == len(H.levels)
    if not os.path.exists(GOLDEN):
        h.close()
        pytest.skip("no stored oracle count (tests/golden/make_golden.py varcoef2048_mg)")
    g = json.load(open(GOLDEN))
    assert g["omega"] == om
    bd = torch.tensor(p["b"], device="cuda")
    x = torch.zeros_like(bd)
    res = h.solve(nd.PCG, nd.PREC_MG, bd, x, rtol=1e-8, maxit=2000, omega=om)
    h.close()
    assert res["relres"] <= 1e-8
    assert abs(res["iters"] - g["iters"]) <= 1, (res, g)


CASES3 = [
    ((40, 36, 30), (2, 2, 2), 0.9, 51),   # 3 levels
    ((33, 31, 29), (3, 2, 2), 0.85, 52),  # odd sides, interior start vertices
    ((64, 20, 18), (4, 1, 1), 0.9, 53),   # slabs
]


def _matrix3(n, seed):
    """SPD 7-point matrix from random face conductances (lognormal)."""
    g = np.random.default_rng(seed)
    nx, ny, nz = n
    N = nx * ny * nz
    d = np.zeros((7, N))
    idx = np.arange(N).reshape(nz, ny, nx)
    for a, (lo, hi) in enumerate(((1, 2), (3, 4), (5, 6))):
        ax = 2 - a
        sl_lo, sl_hi = [slice(None)] * 3, [slice(None)] * 3
        sl_lo[ax], sl_hi[ax] = slice(0, -1), slice(1, None)
        i_lo, i_hi = idx[tuple(sl_lo)].ravel(), idx[tuple(sl_hi)].ravel()
        k = np.exp(0.5 * g.standard_normal(i_lo.size))
        d[hi, i_lo] = -k
        d[lo, i_hi] = -k
    d[0] = -d[1:].sum(axis=0) + 0.01
    return d


@pytest.mark.parametrize("n,sub,om,seed", CASES3)
def test_vcycle3_matches_oracle(nd, n, sub, om, seed):
    import torch
    d = _matrix3(n, seed)
    N = int(np.prod(n))
    r = np.random.default_rng(seed).standard_normal(N)
    H = M.Hierarchy3(n, d, sub, om)
    want = H.vcycle(r)
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    rd = torch.tensor(r, device="cuda")
    z = torch.empty_like(rd)
    h.mg_apply(om, rd, z)
    assert h.mg_levels() == len(H.levels)
    err = np.abs(z.cpu().numpy() - want).max() / np.abs(want).max()
    h.close()
    assert err <= VTOL, err


def test_pcg_mg3_matches_oracle_count(nd):
    import torch
    n, sub, om = (40, 36, 30), (2, 2, 2), 0.9
    d = _matrix3(n, 54)
    b = W.uniform_rhs(int(np.prod(n)), 55)
    H = M.Hierarchy3(n, d, sub, om)
    xr, info = M.pcg(H, b, 1e-8, 300)
    assert info["status"] == 0
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    bd = torch.tensor(b, device="cuda")
    x = torch.zeros_like(bd)
    res = h.solve(nd.PCG, nd.PREC_MG, bd, x, rtol=1e-8, maxit=300, omega=om)
    h.close()
    assert res["relres"] <= 1e-8
    assert abs(res["iters"] - info["iters"]) <= 1, (res, info)


def test_full_size_vcycle3_and_count(nd):
    """256^3 Poisson with 8 x 8 x 8 subdomains, the configuration bench.py's
    3D multigrid line times: one V-cycle element by element against the
    oracle's, and the PCG count against the stored oracle count."""
    import torch
    p = W.poisson3d_problem()
    om = 0.9
    H = M.Hierarchy3(p["n"], p["diags"], p["sub"], om)
    want = H.vcycle(p["b"])
    h = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], "fp64")
    bd = torch.tensor(p["b"], device="cuda")
    z = torch.empty_like(bd)
    h.mg_apply(om, bd, z)
    err = np.abs(z.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= VTOL, err
    assert h.mg_levels() == len(H.levels)
    del H
    path = os.path.join(os.path.dirname(__file__), "golden", "poisson3d256_mg.json")
    if not os.path.exists(path):
        h.close()
        pytest.skip("no stored oracle count (tests/golden/make_golden.py poisson3d256_mg)")
    g = json.load(open(path))
    assert g["omega"] == om
    x = torch.zeros_like(bd)
    res = h.solve(nd.PCG, nd.PREC_MG, bd, x, rtol=1e-8, maxit=500, omega=om)
    h.close()
    assert res["relres"] <= 1e-8
    assert abs(res["iters"] - g["iters"]) <= 1, (res, g)
