"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances:
  fp64 sweeps / applies: max |x - x_oracle| <= 1e-12 max |x_oracle|
  fp32 sweeps:           <= 2e-5  (unit roundoff 6e-8, ~30x growth along the wavefront)
  fp32 + fp16 diagonals: <= 2e-3  (coefficients rounded to 2^-11)
  iteration counts:      SSOR-PCG and the stationary iteration within 1 of the
                         oracle; BiCGSTAB and unpreconditioned CG inside the
                         oracle's own envelope
                         (its count under 1e-15 relative perturbations of b,
                         widened by 1), because BiCGSTAB's count at 1e-8 moves
                         by several iterations under rounding-level changes.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _rand_matrix(n, seed, stencil=5):
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.2, 1.0, size=(stencil, N))
    d = W._zero_outside(d, (n[0], n[1]), stencil)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


def oracle_envelope(ref, method, prec, mode, b, rtol=1e-8, maxit=20000, k=8, eps=1e-15):
    """min/max iteration count of the oracle over k rounding-level
    perturbations of b (and b itself), widened by one."""
    g = np.random.default_rng(12345)
    counts = []
    for j in range(k + 1):
        bb = b if j == 0 else b * (1.0 + eps * g.standard_normal(b.shape))
        _, info = ref.solve(method, prec, mode, 1.0, rtol, maxit, bb)
        counts.append(info["iters"])
    return min(counts) - 1, max(counts) + 1


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))


SWEEP_CASES = [
    ((13, 11), (2, 2)),      # ragged, one band
    ((40, 37), (3, 2)),
    ((70, 200), (2, 1)),     # subdomain of 200 rows: 7 bands, two slabs (CTA handoff)
    ((9, 300), (2, 2)),      # narrow, tall
    ((64, 64), (2, 2)),
    ((129, 260), (4, 2)),
    ((300, 20), (7, 1)),
    ((8, 8), (8, 8)),        # every cell a subdomain: twins and corners everywhere
    ((1, 50), (1, 5)),       # one column
    ((50, 1), (5, 1)),       # one row
    ((33, 33), (1, 1)),
]


@pytest.mark.parametrize("n,sub", SWEEP_CASES)
def test_sor_sweep_fp64_matches_oracle(nd, n, sub):
    d = _rand_matrix(n, 1)
    N = n[0] * n[1]
    g = np.random.default_rng(2)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    om = g.uniform(0.6, 1.8, 4)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    ref = oracle.Problem(2, n, 5, d, sub)
    xb, xo = _t(b), _t(u)
    for t in range(6):
        xn = _t(np.full(N, np.nan))
        h.sor_sweep(om, t, xb, xo, xn)
        want = ref.sor_sweep(oracle.DECOMPOSED, t, om, b, u)
        assert _rel(xn.cpu().numpy(), want) <= 1e-12, t


@pytest.mark.parametrize("n", [(37, 29), (45, 290), (200, 140)])
def test_natural_sor_sweep_matches_oracle(nd, n):
    d = _rand_matrix(n, 3)
    N = n[0] * n[1]
    g = np.random.default_rng(4)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    h = nd.NDiag(2, n, 5, d, (2, 2), "fp64")
    ref = oracle.Problem(2, n, 5, d, (1, 1))
    xn = _t(np.zeros(N))
    h.sor_sweep(1.3, 0, _t(b), _t(u), xn, mode=nd.NATURAL)
    assert _rel(xn.cpu().numpy(), ref.sor_sweep(oracle.NATURAL, 0, 1.3, b, u)) <= 1e-12


@pytest.mark.parametrize("n,sub,mode", [((40, 37), (3, 2), 1), ((70, 200), (2, 1), 1), ((8, 8), (8, 8), 1),
                                        ((37, 29), (1, 1), 0), ((45, 290), (1, 1), 0), ((129, 260), (4, 2), 1)])
def test_ilu0_apply_fp64_matches_oracle(nd, n, sub, mode):
    d = _rand_matrix(n, 5)
    N = n[0] * n[1]
    r = np.random.default_rng(6).uniform(-1, 1, N)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    h.ilu0_factor(mode)
    ref = oracle.Problem(2, n, 5, d, sub if mode else (1, 1))
    ref.ilu0_factor(mode)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(r), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12


@pytest.mark.parametrize("n,sub,mode", [((13, 11), (2, 2), 1), ((40, 37), (3, 2), 1), ((70, 200), (2, 1), 1),
                                        ((30, 31), (4, 3), 1), ((8, 8), (8, 8), 1), ((45, 90), (1, 1), 0),
                                        ((64, 64), (4, 4), 1)])
def test_ssor_apply_fp64_matches_oracle(nd, n, sub, mode):
    d = _rand_matrix(n, 7)  # nonsymmetric: exercises the transposed coefficients
    N = n[0] * n[1]
    r = np.random.default_rng(8).uniform(-1, 1, N)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    ref = oracle.Problem(2, n, 5, d, sub)
    for om in (1.0, 1.4):
        z = _t(np.zeros(N))
        h.ssor_apply(om, _t(r), z, mode=mode)
        assert _rel(z.cpu().numpy(), ref.ssor_apply(mode, om, r)) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp32_d16", 2e-3)])
def test_fp32_sweeps_within_derived_tolerance(nd, prec, tol):
    import torch
    n, sub = (96, 80), (3, 2)
    alpha = W.smoothed_lognormal_alpha(n[0], n[1], 11)
    d = W.diffusion2d(alpha)
    N = n[0] * n[1]
    g = np.random.default_rng(9)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    h = nd.NDiag(2, n, 5, d, sub, prec)
    ref = oracle.Problem(2, n, 5, d, sub)
    f32 = torch.float32
    xn = _t(np.zeros(N), f32)
    h.sor_sweep(1.2, 0, _t(b, f32), _t(u, f32), xn)
    assert _rel(xn.double().cpu().numpy(), ref.sor_sweep(oracle.DECOMPOSED, 0, 1.2, b, u)) <= tol
    z = _t(np.zeros(N), f32)
    h.ssor_apply(1.0, _t(b, f32), z)
    assert _rel(z.double().cpu().numpy(), ref.ssor_apply(oracle.DECOMPOSED, 1.0, b)) <= tol
    h.ilu0_factor(nd.DECOMPOSED)
    ref.ilu0_factor(oracle.DECOMPOSED)
    h.ilu0_apply(_t(b, f32), z)
    assert _rel(z.double().cpu().numpy(), ref.ilu0_apply(b)) <= tol


SOLVE_CASES = [
    ("bicgstab", "ilu0", 1, (96, 96), (3, 3)),
    ("bicgstab", "ilu0", 0, (96, 96), (1, 1)),
    ("pcg", "ssor", 1, (96, 96), (4, 2)),
    ("pcg", "ssor", 0, (96, 96), (1, 1)),
    ("pcg", "none", 1, (64, 50), (2, 2)),
]


@pytest.mark.parametrize("method,prec,mode,n,sub", SOLVE_CASES)
def test_fp64_solvers_match_oracle_iteration_counts(nd, method, prec, mode, n, sub):
    alpha = W.smoothed_lognormal_alpha(n[0], n[1], 13)
    d = W.diffusion2d(alpha)
    b = W.uniform_rhs(n[0] * n[1], 14)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    ref = oracle.Problem(2, n, 5, d, sub)
    M = {"pcg": (nd.PCG, oracle.PCG), "bicgstab": (nd.BICGSTAB, oracle.BICGSTAB)}[method]
    P = {"none": (nd.PREC_NONE, oracle.PREC_NONE), "ssor": (nd.PREC_SSOR, oracle.PREC_SSOR),
         "ilu0": (nd.PREC_ILU0, oracle.PREC_ILU0)}[prec]
    if prec == "ilu0":
        h.ilu0_factor(mode)
    x = _t(np.zeros(n[0] * n[1]))
    info = h.solve(M[0], P[0], _t(b), x, rtol=1e-8, maxit=5000, omega=1.0, mode=mode)
    xr, oinfo = ref.solve(M[1], P[1], mode, 1.0, 1e-8, 5000, b)
    assert info["relres"] <= 1e-8
    if method == "pcg" and prec == "ssor":
        assert abs(info["iters"] - oinfo["iters"]) <= 1, (info, oinfo)
    else:  # BiCGSTAB, and CG without a preconditioner, are rounding-sensitive
        lo, hi = oracle_envelope(ref, M[1], P[1], mode, b)
        assert lo <= info["iters"] <= hi, (info, oinfo, lo, hi)
    # forward error <= cond(A) x (sum of the two relative residuals); cond(A) <= 5e3 here
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-4 * np.linalg.norm(xr)


def test_poisson64_stationary_iteration_counts(nd):
    p = W.poisson64_problem()
    gold = json.load(open(os.path.join(GOLDEN, "poisson64.json")))
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    for name, mode in (("natural", nd.NATURAL), ("decomposed", nd.DECOMPOSED)):
        x = _t(np.zeros(64 * 64))
        info = h.solve(nd.STATIONARY, nd.PREC_NONE, _t(p["b"]), x, rtol=1e-8, maxit=10000,
                       omega=p["omega"], mode=mode)
        assert info["relres"] <= 1e-8
        assert abs(info["iters"] - gold[name]["iters"]) <= 1, (name, info, gold[name])


@pytest.mark.parametrize("prec", ["fp32", "fp32_d16"])
@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_fp32_refinement_reaches_1e8(nd, prec, method):
    n, sub = (128, 96), (4, 3)
    alpha = W.smoothed_lognormal_alpha(n[0], n[1], 15)
    d = W.diffusion2d(alpha)
    b = W.uniform_rhs(n[0] * n[1], 16)
    h = nd.NDiag(2, n, 5, d, sub, prec)
    if method == "pcg":
        info = h.solve(nd.PCG, nd.PREC_SSOR, _t(b), x := _t(np.zeros(n[0] * n[1])), rtol=1e-8, maxit=20000)
    else:
        h.ilu0_factor(nd.DECOMPOSED)
        info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(b), x := _t(np.zeros(n[0] * n[1])), rtol=1e-8,
                       maxit=20000)
    assert info["relres"] <= 1e-8, info
    ref = oracle.Problem(2, n, 5, d, sub)
    xr, _ = ref.solve(oracle.PCG, oracle.PREC_SSOR, oracle.DECOMPOSED, 1.0, 1e-12, 20000, b)
    err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= 1e-5, err  # forward error bound ~ cond(A) * 1e-8


def test_host_pointers_through_the_abi(nd):
    n, sub = (48, 40), (2, 2)
    d = W.diffusion2d(W.smoothed_lognormal_alpha(n[0], n[1], 17))
    b = W.uniform_rhs(n[0] * n[1], 18)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    x = np.zeros(n[0] * n[1])
    info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, b, x, rtol=1e-8)
    A_x = oracle.Problem(2, n, 5, d, sub).matvec(x)
    assert np.linalg.norm(b - A_x) <= 1e-8 * np.linalg.norm(b) * 1.0001, info


def test_invalid_arguments_are_rejected(nd):
    d = _rand_matrix((10, 10), 1)
    with pytest.raises(nd.NdiagError):
        nd.NDiag(2, (10, 10), 5, d, (11, 1), "fp64")
    h = nd.NDiag(2, (10, 10), 5, d, (2, 2), "fp64")
    x = _t(np.zeros(100))
    with pytest.raises(nd.NdiagError):
        h.sor_sweep(1.0, 0, x, x, x)  # x_new aliases x_old
    with pytest.raises(nd.NdiagError):
        h.ilu0_apply(x, _t(np.zeros(100)))  # before ilu0_factor
    with pytest.raises(nd.NdiagError):
        h.ssor_apply(2.5, x, _t(np.zeros(100)))


# ---------------------------------------------------------------------------
# Full size, in the launch configuration bench.py times (2048^2, 16 x 16)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big(nd):
    p = W.varcoef2d_problem(2048, 16)
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    ref = oracle.Problem(2, p["n"], 5, p["diags"], p["sub"])
    return p, h, ref


def test_full_size_sweeps_match_oracle(nd, big):
    p, h, ref = big
    N = 2048 * 2048
    u = W.uniform_rhs(N, 77)
    xb, xo, xn = _t(p["b"]), _t(u), _t(np.zeros(N))
    for t in (0, 1, 2, 3):
        h.sor_sweep(1.5, t, xb, xo, xn)
        assert _rel(xn.cpu().numpy(), ref.sor_sweep(oracle.DECOMPOSED, t, 1.5, p["b"], u)) <= 1e-12


def test_full_size_ilu_apply_matches_oracle(nd, big):
    p, h, ref = big
    h.ilu0_factor(nd.DECOMPOSED)
    ref.ilu0_factor(oracle.DECOMPOSED)
    z = _t(np.zeros(2048 * 2048))
    h.ilu0_apply(_t(p["b"]), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(p["b"])) <= 1e-12


def test_full_size_solve_meets_tolerance_and_oracle_count(nd, big):
    p, h, _ = big
    h.ilu0_factor(nd.DECOMPOSED)
    x = _t(np.zeros(2048 * 2048))
    info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(p["b"]), x, rtol=1e-8, maxit=20000)
    assert info["relres"] <= 1e-8
    # BiCGSTAB's count moves under rounding (see the module docstring): the
    # oracle's own counts for this workload, unperturbed and under seven 1e-15
    # relative perturbations of b, span the envelope (stored by
    # tests/golden/make_golden.py), widened by 1.
    gold = json.load(open(os.path.join(GOLDEN, "varcoef2048.json")))["decomposed"]
    env = json.load(open(os.path.join(GOLDEN, "varcoef2048_envelope.json")))
    lo, hi = min(env["min"], gold["iters"]) - 1, max(env["max"], gold["iters"]) + 1
    assert lo <= info["iters"] <= hi, (info, lo, hi)


@pytest.mark.parametrize("shape,stencil,sub", [((96, 80), 5, (3, 2)), ((31, 17), 5, (1, 1)),
                                               ((24, 20, 18), 7, (2, 2, 2)), ((40, 33), 9, (2, 3))])
def test_residual_matches_the_oracle_matvec(nd, shape, stencil, sub):
    """ndiag_residual: r = b - A x element by element against b minus the
    oracle's matrix-vector product, and the returned norm against ||r||."""
    dim = len(shape)
    N = int(np.prod(shape))
    if stencil == 9:
        diags = W.convdiff9(shape[0], 4.0, 0.7) if shape[0] == shape[1] else W.embed5in9(
            W.diffusion2d(W.smoothed_lognormal_alpha(shape[0], shape[1], 5)))
    elif dim == 3:
        diags = W.poisson3d(*shape)
    else:
        diags = W.diffusion2d(W.smoothed_lognormal_alpha(shape[0], shape[1], 5))
    b, x = W.uniform_rhs(N, 61), W.uniform_rhs(N, 62)
    h = nd.NDiag(dim, shape, stencil, diags, sub, "fp64")
    r = _t(np.zeros(N))
    nrm = h.residual(_t(b), _t(x), r)
    want = b - oracle.Problem(dim, shape, stencil, diags, sub).matvec(x)
    got = r.cpu().numpy()
    # rounding of a sum of `stencil` products and b, in any order: a few ulp of
    # |b| + |A| |x| per cell
    scale = np.abs(b) + oracle.Problem(dim, shape, stencil, np.abs(diags), sub).matvec(np.abs(x))
    assert np.all(np.abs(got - want) <= 16 * 2.0 ** -53 * scale)
    assert abs(nrm - np.linalg.norm(want)) <= 1e-13 * np.linalg.norm(want)
    h.close()
