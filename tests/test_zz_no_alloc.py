"""ilu0_apply_noalloc against ilu0_apply, through the C ABI.

ilu0_apply_noalloc exists for callers that cannot let the library allocate
device memory during a call; it keeps its scratch in a fixed array inside the
library instead. Its result must equal ilu0_apply's, on consecutive calls
(the array keeps the previous call's contents), including a subdomain split
that needs the slab hand-off words, and it must refuse grids larger than its
array.
"""
import numpy as np
import pytest

from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_3699_gb300 import build, ndiag
    build.build()
    return ndiag


def _t(a):
    import torch
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,sub,mode", [((96, 80), (3, 2), 1),      # one slab per subdomain
                                        ((70, 300), (2, 1), 1),     # 300-row subdomains: slab hand-off
                                        ((40, 290), (1, 1), 0)])    # natural ordering, hand-off
def test_noalloc_apply_equals_ilu0_apply_on_consecutive_calls(nd, n, sub, mode):
    d = W.diffusion2d(W.smoothed_lognormal_alpha(n[0], n[1], 21))
    N = n[0] * n[1]
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    h.ilu0_factor(mode)
    for seed in (22, 23):
        r = _t(W.uniform_rhs(N, seed))
        want, got = _t(np.zeros(N)), _t(np.full(N, np.nan))
        h.ilu0_apply(r, want)
        h.ilu0_apply_noalloc(r, got)
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - w)) <= 1e-12 * np.max(np.abs(w))


def test_noalloc_apply_rejects_grids_beyond_its_array(nd):
    n = (1100, 1000)
    assert n[0] * n[1] > nd.NOALLOC_MAX_CELLS
    d = W.poisson2d(*n)
    h = nd.NDiag(2, n, 5, d, (4, 4), "fp64")
    h.ilu0_factor(nd.DECOMPOSED)
    r = _t(np.ones(n[0] * n[1]))
    with pytest.raises(nd.NdiagError) as e:
        h.ilu0_apply_noalloc(r, r)
    assert e.value.status == nd.EINVAL
