"""Failure detection of the bounded device-side waits, without a GPU fault:
a wait on a word that nothing sets runs out after its bound, the kernel
records NDIAG_ETIMEOUT and returns, the host reads the status, and the same
handle then runs a sweep that still matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_1008_3699_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_handle_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1008_3699_gb300 import build, ndiag as nd
    build.build()
    n, sub = (48, 40), (3, 2)
    d = W.poisson2d(*n)
    N = n[0] * n[1]
    g = np.random.default_rng(5)
    b, u = g.uniform(-1, 1, N), g.uniform(-1, 1, N)
    h = nd.NDiag(2, n, 5, d, sub, "fp64")
    assert h.selftest_wait() == "ETIMEOUT"
    assert "timed out" in h.L.ndiag_last_error().decode()
    xn = torch.zeros(N, dtype=torch.float64, device="cuda")
    h.sor_sweep(1.3, 0, torch.tensor(b, device="cuda"), torch.tensor(u, device="cuda"), xn)
    ref = oracle.Problem(2, n, 5, d, sub).sor_sweep(oracle.DECOMPOSED, 0, 1.3, b, u)
    assert np.max(np.abs(xn.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    info = h.solve(nd.PCG, nd.PREC_SSOR, torch.tensor(b, device="cuda"), x, rtol=1e-8)
    assert info["status"] == "OK" and info["relres"] <= 1e-8
    h.close()
