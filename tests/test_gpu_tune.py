"""Per-direction relaxation of the stationary decomposed SOR iteration
(ndiag_tune_omega) on the 64^2 Poisson workload: the factors found converge to
rel-res 1e-8 in fewer sweeps than the single optimal factor 2/(1+sin(pi/65)),
and the oracle with the same factors takes the same number of sweeps (within
one)."""
import numpy as np
import pytest

import oracle
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


def test_tuned_factors_beat_the_uniform_optimum_and_match_the_oracle(nd):
    import torch
    p = W.poisson64_problem()
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    b = torch.tensor(p["b"], device="cuda")
    x = torch.zeros_like(b)
    uni = h.solve(nd.STATIONARY, nd.PREC_NONE, b, x, rtol=1e-8, maxit=20000, omega=p["omega"])
    om, its = h.tune_omega(b, rtol=1e-8, maxit=20000, budget=60, omega=p["omega"])
    h.close()
    assert len(om) == 4 and all(0.0 < w < 2.0 for w in om)
    assert its < uni["iters"], (its, uni, om)
    ref = oracle.Problem(2, (64, 64), 5, p["diags"], (2, 2))
    _, info = ref.solve(oracle.STATIONARY, oracle.PREC_NONE, oracle.DECOMPOSED, om, 1e-8, 20000, p["b"])
    assert abs(info["iters"] - its) <= 1, (info, its)
    assert info["relres"] <= 1e-8


def test_bad_factors_are_refused(nd):
    import torch
    p = W.poisson64_problem()
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    b = torch.tensor(p["b"], device="cuda")
    with pytest.raises(nd.NdiagError):
        h.tune_omega(b, omega=[1.0, 2.5, 1.0, 1.0])
    h.close()
