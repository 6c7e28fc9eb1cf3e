"""Solve server (serve_submit / serve_poll): requests of different kinds
(9-point ILU(0)-BiCGSTAB, 3D SSOR-PCG, fp32 + refinement) run concurrently;
each reaches relative residual 1e-8 (oracle matrix-vector product on the
host) and its result is bit for bit the same alone and in the mix; admission
by the memory budget serialises the solves when the budget is small.
"""
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


def _requests(nd):
    n9 = 40
    r9 = dict(dim=2, n=(n9, n9, 1), stencil=9, diags=W.convdiff9(n9, 6.0, 1.1), b=W.uniform_rhs(n9 * n9, 5),
              sub=(2, 2, 1))
    n3 = 12
    r3 = dict(dim=3, n=(n3, n3, n3), stencil=7, diags=W.poisson3d(n3, n3, n3), b=W.uniform_rhs(n3 ** 3, 6),
              sub=(2, 2, 2))
    n5 = 50
    r5 = dict(dim=2, n=(n5, n5, 1), stencil=5, diags=W.diffusion2d(W.loguniform_alpha(n5, n5, 7)),
              b=W.uniform_rhs(n5 * n5, 8), sub=(2, 2, 1))
    n4 = 16
    r4 = dict(dim=3, n=(n4, n4, n4), stencil=7, diags=W.poisson3d(n4, n4, n4), b=W.uniform_rhs(n4 ** 3, 9),
              sub=(2, 2, 2))
    return [(r9, dict(method=nd.BICGSTAB, precond=nd.PREC_ILU0, precision="fp64")),
            (r3, dict(method=nd.PCG, precond=nd.PREC_SSOR, precision="fp64")),
            (r5, dict(method=nd.PCG, precond=nd.PREC_SSOR, precision="fp32")),
            (r4, dict(method=nd.PCG, precond=nd.PREC_SSOR, precision="fp32"))]


def _relres(p, x):
    ref = oracle.Problem(p["dim"], p["n"][: p["dim"]], p["stencil"], p["diags"], (1, 1, 1))
    return np.linalg.norm(p["b"] - ref.matvec(x)) / np.linalg.norm(p["b"])


def test_mixed_requests_converge_and_match_alone(nd):
    reqs = _requests(nd)
    S = nd.Server(slots=4)
    tickets = [S.submit(p, **kw) for p, kw in reqs]
    mixed = [S.wait(t) for t in tickets]
    st = S.stats()
    S.close()
    for (p, _), (res, x) in zip(reqs, mixed):
        assert res["status"] == "OK", res
        assert res["relres"] <= 1e-8
        assert _relres(p, x) <= 1e-8
        assert res["latency_s"] >= res["run_s"] > 0
    assert st["solved"] == len(reqs)
    # each request alone
    for (p, kw), (_, xm) in zip(reqs, mixed):
        A = nd.Server(slots=1)
        res, xa = A.wait(A.submit(p, **kw))
        A.close()
        assert np.array_equal(xa, xm)


def test_small_budget_serialises_admission(nd):
    reqs = _requests(nd)
    S = nd.Server(slots=3, mem_budget=1)
    tickets = [S.submit(p, **kw) for p, kw in reqs]
    out = [S.wait(t) for t in tickets]
    st = S.stats()
    S.close()
    assert all(r["status"] == "OK" for r, _ in out)
    assert st["max_running"] == 1
    assert st["in_use_bytes"] == 0


def test_bad_request_is_refused(nd):
    S = nd.Server(slots=1)
    p = dict(dim=3, n=(4, 4, 4), stencil=9, diags=np.zeros((9, 64)), b=np.zeros(64))
    with pytest.raises(nd.NdiagError):
        S.submit(p)
    S.close()
