"""GPU parity of the 3D 7-point path (level sweep, sweep3d.cu) against the CPU
oracle, through the C ABI. Tolerances as in test_gpu_parity.py: fp64 sweeps and
applies to 1e-12 relative (max norm), fp32 to 2e-5, SSOR-PCG iteration counts
within 1 of the oracle, fp32 + fp64 refinement to relative residual 1e-8.

Grids cover even and uneven splits, one-cell-thick subdomains (every cell on
a start face, so corners, edges and faces meet), and every phase of the
eight-sweep 3D schedule.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [((12, 10, 9), (2, 2, 2)), ((13, 11, 7), (3, 2, 2)), ((5, 6, 7), (5, 3, 2)), ((16, 16, 16), (2, 2, 2))]


@pytest.fixture(scope="module")
def nd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_3699_gb300 import build, ndiag
    build.build()
    return ndiag


def _t(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float64, device="cuda")


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


def _nonsym7(n, seed):
    """Random diagonally dominant nonsymmetric 7-point matrix."""
    g = np.random.default_rng(seed)
    N = n[0] * n[1] * n[2]
    d = -g.uniform(0.2, 1.0, size=(7, N))
    d = W._zero_outside(d, n, 7)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def _sym7(n, seed):
    """Symmetric positive definite 7-point matrix from random face conductances."""
    g = np.random.default_rng(seed)
    nx, ny, nz = n
    N = nx * ny * nz
    d = np.zeros((7, N))
    idx = np.arange(N).reshape(nz, ny, nx)
    for a, (lo, hi) in enumerate(((1, 2), (3, 4), (5, 6))):
        ax = 2 - a  # numpy axis of grid axis a
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        i_lo = idx[tuple(sl_lo)].ravel()
        i_hi = idx[tuple(sl_hi)].ravel()
        k = g.uniform(0.5, 2.0, i_lo.size)
        d[hi, i_lo] = -k  # i_lo's neighbour at +a
        d[lo, i_hi] = -k  # i_hi's neighbour at -a
    d[0] = -d[1:].sum(axis=0) + 0.05
    return d


@pytest.mark.parametrize("n,sub", CASES)
def test_sor_sweep3d_all_phases_fp64(nd, n, sub):
    d = _nonsym7(n, 31)
    N = int(np.prod(n))
    g = np.random.default_rng(32)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    om = g.uniform(0.8, 1.6, 8)
    ref = oracle.Problem(3, n, 7, d, sub)
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    xn = _t(np.zeros(N))
    for mode in (nd.DECOMPOSED, nd.NATURAL):
        for t in range(8):
            h.sor_sweep(om, t, _t(b), _t(u), xn, mode=mode)
            want = ref.sor_sweep(mode, t, om, b, u)
            assert _rel(xn.cpu().numpy(), want) <= 1e-12, (mode, t)
    h.close()


@pytest.mark.parametrize("n,sub", CASES)
@pytest.mark.parametrize("mode", [1, 0])
def test_ilu0_apply3d_fp64(nd, n, sub, mode):
    d = _nonsym7(n, 41)
    N = int(np.prod(n))
    r = np.random.default_rng(42).uniform(-1, 1, N)
    ref = oracle.Problem(3, n, 7, d, sub)
    ref.ilu0_factor(mode)
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    h.ilu0_factor(mode)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(r), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()


@pytest.mark.parametrize("n,sub", CASES)
@pytest.mark.parametrize("mode", [1, 0])
def test_ssor_apply3d_fp64(nd, n, sub, mode):
    d = _sym7(n, 51)
    N = int(np.prod(n))
    r = np.random.default_rng(52).uniform(-1, 1, N)
    ref = oracle.Problem(3, n, 7, d, sub)
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    z = _t(np.zeros(N))
    for om in (1.0, 1.3):
        h.ssor_apply(om, _t(r), z, mode=mode)
        assert _rel(z.cpu().numpy(), ref.ssor_apply(mode, om, r)) <= 1e-12, om
    h.close()


def test_pcg_ssor3d_iterations_match_oracle(nd):
    n, sub = (16, 16, 16), (2, 2, 2)
    d = _sym7(n, 61)
    N = int(np.prod(n))
    b = np.random.default_rng(62).uniform(-1, 1, N)
    ref = oracle.Problem(3, n, 7, d, sub)
    _, want = ref.solve(oracle.PCG, oracle.PREC_SSOR, oracle.DECOMPOSED, 1.0, 1e-8, 2000, b)
    h = nd.NDiag(3, n, 7, d, sub, "fp64")
    x = _t(np.zeros(N))
    info = h.solve(nd.PCG, nd.PREC_SSOR, _t(b), x, rtol=1e-8, maxit=2000)
    assert info["relres"] <= 1e-8
    assert abs(info["iters"] - want["iters"]) <= 1, (info, want)
    h.close()


def test_fp32_refinement3d_reaches_fp64_tolerance(nd):
    import torch
    n, sub = (24, 20, 18), (3, 2, 2)
    d = W.poisson3d(*n)
    N = int(np.prod(n))
    b = W.uniform_rhs(N, 1003)
    ref = oracle.Problem(3, n, 7, d, sub)
    xr, _ = ref.solve(oracle.PCG, oracle.PREC_SSOR, oracle.DECOMPOSED, 1.0, 1e-10, 5000, b)
    h = nd.NDiag(3, n, 7, d, sub, "fp32")
    x = _t(np.zeros(N))
    info = h.solve(nd.PCG, nd.PREC_SSOR, _t(b), x, rtol=1e-8, maxit=5000)
    assert info["relres"] <= 1e-8
    r = b - ref.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    # forward error against the fp64 oracle solution (kappa of this Poisson grid ~ 3e2)
    assert _rel(x.cpu().numpy(), xr) <= 1e-5
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp32_d16", 2e-3)])
def test_sweeps3d_reduced_precision(nd, prec, tol):
    import torch
    n, sub = (13, 11, 7), (3, 2, 2)
    d = _sym7(n, 71)
    N = int(np.prod(n))
    g = np.random.default_rng(72)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    ref = oracle.Problem(3, n, 7, d, sub)
    h = nd.NDiag(3, n, 7, d, sub, prec)
    f32 = torch.float32
    xn = _t(np.zeros(N), f32)
    h.sor_sweep(1.2, 3, _t(b, f32), _t(u, f32), xn)
    assert _rel(xn.cpu().numpy(), ref.sor_sweep(oracle.DECOMPOSED, 3, 1.2, b, u)) <= tol
    z = _t(np.zeros(N), f32)
    h.ssor_apply(1.0, _t(b, f32), z)
    assert _rel(z.cpu().numpy(), ref.ssor_apply(oracle.DECOMPOSED, 1.0, b)) <= tol
    h.ilu0_factor(nd.DECOMPOSED)
    ref.ilu0_factor(oracle.DECOMPOSED)
    h.ilu0_apply(_t(b, f32), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(b)) <= tol
    h.close()


def test_full_size_applies_match_oracle(nd):
    """The 256^3 Poisson workload with 8 x 8 x 8 subdomains, in the launch
    configuration the benchmark times: the fp64 SSOR apply and the decomposed
    ILU(0) apply element by element against the oracle (1e-12), and the fp32
    SSOR apply (2e-5)."""
    import torch
    p = W.poisson3d_problem()
    N = int(np.prod(p["n"]))
    r = p["b"]
    ref = oracle.Problem(3, p["n"], 7, p["diags"], p["sub"])
    want = ref.ssor_apply(oracle.DECOMPOSED, 1.0, r)
    h = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], "fp64")
    z = _t(np.zeros(N))
    h.ssor_apply(1.0, _t(r), z)
    assert _rel(z.cpu().numpy(), want) <= 1e-12
    h.ilu0_factor(nd.DECOMPOSED)
    h.ilu0_apply(_t(r), z)
    ref.ilu0_factor(oracle.DECOMPOSED)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()
    h32 = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], "fp32")
    z32 = _t(np.zeros(N), torch.float32)
    h32.ssor_apply(1.0, _t(r, torch.float32), z32)
    assert _rel(z32.cpu().numpy(), want) <= 2e-5
    h32.close()


WAVE_CASES = [((12, 10, 9), (2, 2, 2)), ((13, 11, 7), (3, 2, 2)), ((5, 6, 7), (5, 3, 2)), ((64, 64, 64), (2, 2, 2)),
              ((40, 33, 35), (1, 1, 1)), ((70, 20, 66), (2, 1, 2)), ((9, 40, 12), (1, 1, 1))]


@pytest.mark.parametrize("n,sub", WAVE_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_wavefront_walk3d_matches_the_level_walk_and_the_oracle(nd, n, sub, prec):
    """The 3D one-cell walk as a wavefront (warp per plane, lane per row,
    shared ring between planes) against the level walk (1e-13 fp64 / 1e-6
    fp32) and the oracle (1e-12 / 2e-5): ILU(0) apply (forward and reverse
    phase) and SSOR apply (forward and transposed passes), on uneven, one-cell
    thick, one-subdomain and 32-plane subdomains; subdomains with more than 32
    rows along y or z take the level walk."""
    import torch
    d = _nonsym7(n, 401 + sub[0])
    ds = _sym7(n, 402 + sub[1])
    N = n[0] * n[1] * n[2]
    r = np.random.default_rng(403).uniform(-1, 1, N)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol_o, tol_k = (1e-12, 1e-13) if prec == "fp64" else (2e-5, 1e-6)
    ref = oracle.Problem(3, n, 7, d, sub)
    ref.ilu0_factor(oracle.DECOMPOSED)
    want_ilu = ref.ilu0_apply(r)
    want_ssor = oracle.Problem(3, n, 7, ds, sub).ssor_apply(oracle.DECOMPOSED, 1.0, r)
    got = {}
    for wave in (True, False):
        h = nd.NDiag(3, n, 7, d, sub, prec)
        h.set_wavefront(wave)
        h.ilu0_factor(nd.DECOMPOSED)
        z = _t(np.zeros(N), dt)
        h.ilu0_apply(_t(r, dt), z)
        h.close()
        hs = nd.NDiag(3, n, 7, ds, sub, prec)
        hs.set_wavefront(wave)
        zs = _t(np.zeros(N), dt)
        hs.ssor_apply(1.0, _t(r, dt), zs)
        hs.close()
        got[wave] = (z.cpu().numpy().astype(np.float64), zs.cpu().numpy().astype(np.float64))
    assert _rel(got[True][0], want_ilu) <= tol_o
    assert _rel(got[True][1], want_ssor) <= tol_o
    assert _rel(got[True][0], got[False][0]) <= tol_k
    assert _rel(got[True][1], got[False][1]) <= tol_k
