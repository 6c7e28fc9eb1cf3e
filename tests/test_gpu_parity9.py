"""GPU parity of the 2D 9-point path (level sweep with x-interface lockstep,
sweep9.cu) against the CPU oracle, through the C ABI: SOR sweeps of every
phase and the natural ordering, the decomposed D-ILU factor and apply to 1e-12
(fp64), fp32 sweeps to 2e-5, an ILU(0)-BiCGSTAB solve of the 9-point
convection-diffusion operator inside the oracle's iteration envelope, and the
natural-order true ILU(0) (modified off-diagonals): apply to 1e-12 / 2e-5,
solve count inside the oracle's envelope, zero pivot reported.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [((20, 17), (2, 2)), ((33, 25), (3, 2)), ((9, 12), (9, 4)), ((40, 40), (4, 4))]


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


def _rand9(n, seed):
    g = np.random.default_rng(seed)
    N = n[0] * n[1]
    d = -g.uniform(0.1, 0.8, size=(9, N))
    d = W._zero_outside(d, (n[0], n[1]), 9)
    d[0] = -d[1:].sum(axis=0) + g.uniform(0.05, 0.5, N)
    return d


@pytest.mark.parametrize("n,sub", CASES)
def test_sor_sweep9_all_phases_fp64(nd, n, sub):
    d = _rand9(n, 91)
    N = n[0] * n[1]
    g = np.random.default_rng(92)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    om = g.uniform(0.8, 1.6, 4)
    ref = oracle.Problem(2, n, 9, d, sub)
    h = nd.NDiag(2, n, 9, d, sub, "fp64")
    xn = _t(np.zeros(N))
    for mode in (nd.DECOMPOSED, nd.NATURAL):
        for t in range(4):
            h.sor_sweep(om, t, _t(b), _t(u), xn, mode=mode)
            want = ref.sor_sweep(mode, t, om, b, u)
            assert _rel(xn.cpu().numpy(), want) <= 1e-12, (mode, t)
    h.close()


@pytest.mark.parametrize("n,sub", CASES)
def test_dilu_apply9_fp64(nd, n, sub):
    d = _rand9(n, 93)
    N = n[0] * n[1]
    r = np.random.default_rng(94).uniform(-1, 1, N)
    ref = oracle.Problem(2, n, 9, d, sub)
    ref.ilu0_factor(oracle.DECOMPOSED)
    h = nd.NDiag(2, n, 9, d, sub, "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(r), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()


def test_sweeps9_fp32(nd):
    import torch
    n, sub = (33, 25), (3, 2)
    d = _rand9(n, 95)
    N = n[0] * n[1]
    g = np.random.default_rng(96)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    ref = oracle.Problem(2, n, 9, d, sub)
    h = nd.NDiag(2, n, 9, d, sub, "fp32")
    f32 = torch.float32
    xn = _t(np.zeros(N), f32)
    h.sor_sweep(1.1, 2, _t(b, f32), _t(u, f32), xn)
    assert _rel(xn.cpu().numpy(), ref.sor_sweep(oracle.DECOMPOSED, 2, 1.1, b, u)) <= 2e-5
    h.ilu0_factor(nd.DECOMPOSED)
    ref.ilu0_factor(oracle.DECOMPOSED)
    z = _t(np.zeros(N), f32)
    h.ilu0_apply(_t(b, f32), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(b)) <= 2e-5
    h.close()


def test_bicgstab_dilu9_convdiff_in_oracle_envelope(nd):
    n, sub = 48, (3, 3)
    d = W.convdiff9(n, 7.0, 0.6)
    N = n * n
    b = W.uniform_rhs(N, 1005)
    ref = oracle.Problem(2, (n, n), 9, d, sub)
    ref.ilu0_factor(oracle.DECOMPOSED)
    counts = []
    g = np.random.default_rng(12345)
    for j in range(7):
        bb = b if j == 0 else b * (1.0 + 1e-15 * g.standard_normal(N))
        _, info = ref.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.DECOMPOSED, 1.0, 1e-8, 5000, bb)
        counts.append(info["iters"])
    h = nd.NDiag(2, (n, n), 9, d, sub, "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    x = _t(np.zeros(N))
    info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(b), x, rtol=1e-8, maxit=5000)
    assert info["relres"] <= 1e-8
    assert min(counts) - 1 <= info["iters"] <= max(counts) + 1, (info, counts)
    r = b - ref.matvec(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    h.close()


def test_nine_point_ssor_is_refused(nd):
    n = (12, 10)
    d = _rand9(n, 97)
    h = nd.NDiag(2, n, 9, d, (2, 2), "fp64")
    z = _t(np.zeros(120))
    with pytest.raises(nd.NdiagError):
        h.ssor_apply(1.0, _t(np.ones(120)), z)
    h.close()


@pytest.mark.parametrize("n", [(20, 17), (33, 25), (9, 12), (1, 7), (7, 1), (2, 5), (300, 40)])
def test_natural_ilu0_apply9_fp64(nd, n):
    # true ILU(0) (modified off-diagonals) in natural order against the oracle's IKJ factor
    d = _rand9(n, 98)
    N = n[0] * n[1]
    r = np.random.default_rng(99).uniform(-1, 1, N)
    ref = oracle.Problem(2, n, 9, d, (1, 1))
    ref.ilu0_factor(oracle.NATURAL)
    h = nd.NDiag(2, n, 9, d, (2, 1) if n[0] > 1 else (1, 1), "fp64")
    h.ilu0_factor(nd.NATURAL)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(r), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()


def test_natural_ilu0_9_fp32_and_solve(nd):
    import torch
    n = 48
    d = W.convdiff9(n, 7.0, 0.6)
    N = n * n
    b = W.uniform_rhs(N, 1007)
    ref = oracle.Problem(2, (n, n), 9, d, (1, 1))
    ref.ilu0_factor(oracle.NATURAL)
    h32 = nd.NDiag(2, (n, n), 9, d, (1, 1), "fp32")
    h32.ilu0_factor(nd.NATURAL)
    z = _t(np.zeros(N), torch.float32)
    h32.ilu0_apply(_t(b, torch.float32), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(b)) <= 2e-5
    h32.close()
    counts = []
    g = np.random.default_rng(4321)
    for j in range(7):
        bb = b if j == 0 else b * (1.0 + 1e-15 * g.standard_normal(N))
        _, info = ref.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.NATURAL, 1.0, 1e-8, 5000, bb)
        counts.append(info["iters"])
    h = nd.NDiag(2, (n, n), 9, d, (3, 3), "fp64")
    h.ilu0_factor(nd.NATURAL)
    x = _t(np.zeros(N))
    info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(b), x, rtol=1e-8, maxit=5000, mode=nd.NATURAL)
    assert info["relres"] <= 1e-8
    assert min(counts) - 1 <= info["iters"] <= max(counts) + 1, (info, counts)
    h.close()


def test_natural_ilu0_9_zero_pivot_is_reported(nd):
    # a row whose elimination cancels its pivot: A = [[1, 1], [1, 1]] on a 2 x 1 grid
    d = np.zeros((9, 2))
    d[0] = 1.0
    d[2, 0] = 1.0   # E of cell 0
    d[1, 1] = 1.0   # W of cell 1
    h = nd.NDiag(2, (2, 1), 9, d, (1, 1), "fp64")
    with pytest.raises(nd.NdiagError):
        h.ilu0_factor(nd.NATURAL)
    h.close()


def test_full_size_dilu_apply9_matches_oracle(nd):
    """The serving line's 9-point operator at 2048^2 with 16 x 16 subdomains
    (paired CTAs): the decomposed D-ILU apply element by element (1e-12)."""
    n = 2048
    d = W.convdiff9(n, 6.0, 1.1)
    N = n * n
    r = W.uniform_rhs(N, 5)
    ref = oracle.Problem(2, (n, n), 9, d, (16, 16))
    ref.ilu0_factor(oracle.DECOMPOSED)
    h = nd.NDiag(2, (n, n), 9, d, (16, 16), "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(r), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()


def test_ilu1_of_a_five_point_matrix_through_the_nine_point_path(nd):
    """Natural ILU(1) of a 5-point matrix: the matrix in 9-point storage (zero
    corners) factored by the natural 9-point ILU(0). Apply to 1e-12 against the
    oracle; PCG count within 1 of the oracle's and below ILU(0)'s."""
    n = (120, 90)
    d5 = W.diffusion2d(W.smoothed_lognormal_alpha(n[0], n[1], 11))
    d9 = W.embed5in9(d5)
    N = n[0] * n[1]
    b = W.uniform_rhs(N, 12)
    ref = oracle.Problem(2, n, 9, d9, (1, 1))
    ref.ilu0_factor(oracle.NATURAL)
    h = nd.NDiag(2, n, 9, d9, (2, 2), "fp64")
    h.ilu0_factor(nd.NATURAL)
    z = _t(np.zeros(N))
    h.ilu0_apply(_t(b), z)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(b)) <= 1e-12
    _, i1 = ref.solve(oracle.PCG, oracle.PREC_ILU0, oracle.NATURAL, 1.0, 1e-8, 2000, b)
    x = _t(np.zeros(N))
    g1 = h.solve(nd.PCG, nd.PREC_ILU0, _t(b), x, rtol=1e-8, maxit=2000, mode=nd.NATURAL)
    h.close()
    assert g1["relres"] <= 1e-8 and abs(g1["iters"] - i1["iters"]) <= 1, (g1, i1)
    h5 = nd.NDiag(2, n, 5, d5, (2, 2), "fp64")
    h5.ilu0_factor(nd.NATURAL)
    x5 = _t(np.zeros(N))
    g0 = h5.solve(nd.PCG, nd.PREC_ILU0, _t(b), x5, rtol=1e-8, maxit=2000, mode=nd.NATURAL)
    h5.close()
    assert g1["iters"] < g0["iters"], (g1, g0)


WAVE_CASES = [((20, 17), (2, 2)), ((33, 25), (3, 2)), ((9, 12), (9, 4)), ((40, 40), (4, 4)), ((37, 29), (1, 1)),
              ((300, 40), (6, 2)), ((130, 129), (1, 1)), ((64, 260), (3, 2)), ((7, 66), (2, 1))]


@pytest.mark.parametrize("n,sub", WAVE_CASES)
@pytest.mark.parametrize("factor", ["dilu", "full"])
def test_wavefront_sweeps9_match_the_oracle_and_the_level_kernel(nd, n, sub, factor):
    """The wavefront kernel (lane = row, packed coefficients, edge warp for the
    coupled start rows, x-pairs through a named barrier) against the oracle's
    apply (1e-12) and against the level kernel (1e-13), forward and backward
    sweeps of both decomposed factors; one-subdomain, one-column, ragged and
    taller-than-four-band partitions (the last fall back to the level kernel)."""
    d = _rand9(n, 301 + sub[0] + sub[1])
    N = n[0] * n[1]
    r = np.random.default_rng(302).uniform(-1, 1, N)
    mode_o = oracle.DECOMPOSED if factor == "dilu" else oracle.DECOMPOSED_FULL
    mode_g = nd.DECOMPOSED if factor == "dilu" else nd.DECOMPOSED_FULL
    ref = oracle.Problem(2, n, 9, d, sub)
    ref.ilu0_factor(mode_o)
    want = ref.ilu0_apply(r)
    out = {}
    for wave in (True, False):
        h = nd.NDiag(2, n, 9, d, sub, "fp64")
        h.set_wavefront(wave)
        h.ilu0_factor(mode_g)
        z = _t(np.zeros(N))
        for _ in range(2):  # the second apply reuses the packed copy
            h.ilu0_apply(_t(r), z)
        h.close()
        out[wave] = z.cpu().numpy()
    assert _rel(out[True], want) <= 1e-12
    assert _rel(out[True], out[False]) <= 1e-13


def test_wavefront_follows_a_new_factor(nd):
    """The packed copy is rebuilt when the coefficient set changes."""
    n, sub = (48, 40), (3, 2)
    d1 = _rand9(n, 311)
    r = np.random.default_rng(313).uniform(-1, 1, n[0] * n[1])
    h = nd.NDiag(2, n, 9, d1, sub, "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    z = _t(np.zeros(n[0] * n[1]))
    h.ilu0_apply(_t(r), z)
    h.ilu0_factor(nd.DECOMPOSED_FULL)
    h.ilu0_apply(_t(r), z)
    ref = oracle.Problem(2, n, 9, d1, sub)
    ref.ilu0_factor(oracle.DECOMPOSED_FULL)
    assert _rel(z.cpu().numpy(), ref.ilu0_apply(r)) <= 1e-12
    h.close()
