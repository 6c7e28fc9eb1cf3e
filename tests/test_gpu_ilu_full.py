"""GPU parity of the decomposed full ILU(0) (ilu0_factor with
DECOMPOSED_FULL: the true ILU(0) of every subdomain's block in its forward-sweep
order, Sec. 5) against the oracle's factor, through the C ABI.

- apply to 1e-12 (fp64) and 2e-5 (fp32) on grids with ragged subdomains, one
  subdomain, one-column subdomains and both paired and unpaired 9-point sweeps;
- a 5-point matrix in 9-point storage: the decomposed ILU(1), to 1e-12;
- 5-point handles: DECOMPOSED_FULL is DECOMPOSED, bit for bit;
- BiCGSTAB's per-iteration record against the oracle's in lockstep, and fewer
  iterations than with D-ILU;
- the 2048^2 9-point convection-diffusion operator with 16 x 16 subdomains;
- a zero pivot is reported.
"""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W
from tests.test_gpu_lockstep import compare, oracle_envelope

pytestmark = pytest.mark.gpu

CASES = [((20, 17), (2, 2)), ((33, 25), (3, 2)), ((9, 12), (9, 4)), ((40, 40), (4, 4)), ((37, 29), (1, 1)),
         ((64, 48), (5, 3)), ((300, 40), (6, 2))]


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


def _apply_pair(nd, n, sub, d, r, precision="fp64", stencil=9):
    import torch
    ref = oracle.Problem(2, n, stencil, d, sub)
    ref.ilu0_factor(oracle.DECOMPOSED_FULL)
    h = nd.NDiag(2, n, stencil, d, sub, precision)
    h.ilu0_factor(nd.DECOMPOSED_FULL)
    dt = torch.float64 if precision == "fp64" else torch.float32
    z = _t(np.zeros(n[0] * n[1]), dt)
    h.ilu0_apply(_t(r, dt), z)
    h.close()
    return z.cpu().numpy().astype(np.float64), ref.ilu0_apply(r)


@pytest.mark.parametrize("n,sub", CASES)
def test_full_ilu_apply9_fp64(nd, n, sub):
    d = _rand9(n, 201 + sub[0])
    r = np.random.default_rng(202).uniform(-1, 1, n[0] * n[1])
    got, want = _apply_pair(nd, n, sub, d, r)
    assert _rel(got, want) <= 1e-12


def test_full_ilu_apply9_fp32(nd):
    n, sub = (33, 25), (3, 2)
    d = _rand9(n, 203)
    r = np.random.default_rng(204).uniform(-1, 1, n[0] * n[1])
    got, want = _apply_pair(nd, n, sub, d, r, "fp32")
    assert _rel(got, want) <= 2e-5


@pytest.mark.parametrize("n,sub", [((48, 40), (3, 2)), ((120, 90), (4, 4))])
def test_decomposed_ilu1_of_a_five_point_matrix(nd, n, sub):
    d5 = W.diffusion2d(W.smoothed_lognormal_alpha(n[0], n[1], 13))
    r = W.uniform_rhs(n[0] * n[1], 14)
    got, want = _apply_pair(nd, n, sub, W.embed5in9(d5), r)
    assert _rel(got, want) <= 1e-12


def test_five_point_full_is_the_decomposed_factor(nd):
    import torch
    n, sub = (50, 44), (3, 4)
    d = W.diffusion2d(W.smoothed_lognormal_alpha(*n, 15))
    r = _t(W.uniform_rhs(n[0] * n[1], 16))
    out = []
    for mode in (nd.DECOMPOSED, nd.DECOMPOSED_FULL):
        h = nd.NDiag(2, n, 5, d, sub, "fp64")
        h.ilu0_factor(mode)
        z = torch.zeros_like(r)
        h.ilu0_apply(r, z)
        h.close()
        out.append(z.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    ref = oracle.Problem(2, n, 5, d, sub)
    ref.ilu0_factor(oracle.DECOMPOSED_FULL)
    assert _rel(out[1], ref.ilu0_apply(r.cpu().numpy())) <= 1e-12


def test_full_ilu_bicgstab_record_in_lockstep(nd):
    n, sub = (96, 96), (3, 2)
    d = W.convdiff9(96, 6.0, 1.1)
    b = W.uniform_rhs(96 * 96, 17)
    kmax = 40
    pb = oracle.Problem(2, n, 9, d, sub)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    ref, dev = oracle_envelope(pb, oracle.BICGSTAB, oracle.PREC_ILU0, oracle.DECOMPOSED, b, kmax, (0, 1, 2, 3))
    h = nd.NDiag(2, n, 9, d, sub, "fp64")
    h.ilu0_factor(nd.DECOMPOSED_FULL)
    x = _t(np.zeros(96 * 96))
    info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(b), x, rtol=1e-8, maxit=kmax, raise_on_noconv=False,
                   history=kmax)
    h.close()
    # the oracle runs all 40 iterations on this operator (rtol 1e-8 is reached later)
    assert len(ref) == kmax
    ok, nrows, worst = compare(info["history"], ref, dev, cols=(0, 1, 2, 3))
    print(f"lockstep full ILU(0): {nrows} rows, worst difference / allowance {worst:.3g}")
    assert ok, (nrows, worst)


def test_full_ilu_needs_fewer_iterations_than_dilu(nd):
    n, sub = 48, (3, 3)
    d = W.convdiff9(n, 6.0, 1.1)
    b = W.uniform_rhs(n * n, 12)
    counts = {}
    for mode in (nd.DECOMPOSED, nd.DECOMPOSED_FULL):
        h = nd.NDiag(2, (n, n), 9, d, sub, "fp64")
        h.ilu0_factor(mode)
        x = _t(np.zeros(n * n))
        info = h.solve(nd.BICGSTAB, nd.PREC_ILU0, _t(b), x, rtol=1e-8, maxit=2000)
        h.close()
        assert info["relres"] <= 1e-8
        counts[mode] = info["iters"]
    pb = oracle.Problem(2, (n, n), 9, d, sub)
    pb.ilu0_factor(oracle.DECOMPOSED_FULL)
    _, oi = pb.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.DECOMPOSED, 1.0, 1e-8, 2000, b)
    assert counts[nd.DECOMPOSED_FULL] < counts[nd.DECOMPOSED], counts
    assert abs(counts[nd.DECOMPOSED_FULL] - oi["iters"]) <= 1, (counts, oi)


def test_full_size_full_ilu_apply9_matches_oracle(nd):
    """2048^2 9-point convection-diffusion, 16 x 16 subdomains (paired CTAs in
    the apply): element by element to 1e-12."""
    n = 2048
    d = W.convdiff9(n, 6.0, 1.1)
    r = W.uniform_rhs(n * n, 5)
    got, want = _apply_pair(nd, (n, n), (16, 16), d, r)
    assert _rel(got, want) <= 1e-12


def test_full_ilu_zero_pivot_is_reported(nd):
    d = np.zeros((9, 2))
    d[0] = 1.0
    d[2, 0] = 1.0
    d[1, 1] = 1.0
    h = nd.NDiag(2, (2, 1), 9, d, (1, 1), "fp64")
    with pytest.raises(nd.NdiagError):
        h.ilu0_factor(nd.DECOMPOSED_FULL)
    h.close()
