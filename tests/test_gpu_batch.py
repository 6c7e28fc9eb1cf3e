"""Batched solves (ndiag_batch_*): every problem of a mixed-size batch reaches
the fp64 relative residual 1e-8 (checked with the oracle's matrix-vector
product on the host), each problem's result is the same alone and in the mix
(per-problem arithmetic is independent of the batch: bit for bit), and the
autotuner picks one of its candidate tiles.
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


def _problems(count, lo, hi, seed):
    return W.batched_problems(count, lo, hi, seed)


def _concat(probs, key="b"):
    return np.concatenate([p[key] for p in probs])


def _true_relres(p, x):
    ref = oracle.Problem(2, p["n"], 5, p["diags"], (1, 1, 1))
    r = p["b"] - ref.matvec(x)
    return np.linalg.norm(r) / np.linalg.norm(p["b"])


def test_batch_solve_reaches_tolerance_and_matches_alone(nd):
    import torch
    probs = _problems(10, 20, 150, 77)
    B = nd.Batch(probs, tile=32)
    b = torch.tensor(_concat(probs), device="cuda")
    x = torch.zeros_like(b)
    infos = B.solve(b, x, rtol=1e-8)
    xs = x.cpu().numpy()
    off = B.offsets
    for k, p in enumerate(probs):
        assert infos[k]["relres"] <= 1e-8, (k, infos[k])
        assert _true_relres(p, xs[off[k]:off[k + 1]]) <= 1e-8
    B.close()
    # alone: bit for bit the same as in the mix
    for k in (0, 3, 9):
        A = nd.Batch([probs[k]], tile=32)
        bk = torch.tensor(probs[k]["b"], device="cuda")
        xk = torch.zeros_like(bk)
        ik = A.solve(bk, xk, rtol=1e-8)
        assert np.array_equal(xk.cpu().numpy(), xs[off[k]:off[k + 1]]), k
        assert ik[0]["iters"] == infos[k]["iters"]
        A.close()


def test_batch_autotune_and_uneven_tiles(nd):
    import torch
    probs = _problems(6, 32, 200, 78)
    B = nd.Batch(probs, tile=[32, 64, 128, 32, 64, 128])
    assert list(B.tiles()) == [32, 64, 128, 32, 64, 128]
    b = torch.tensor(_concat(probs), device="cuda")
    B.autotune(b)
    t = B.tiles()
    assert t[0] in (32, 64, 128) and np.all(t == t[0])
    x = torch.zeros_like(b)
    infos = B.solve(b, x, rtol=1e-8)
    assert all(i["relres"] <= 1e-8 for i in infos)
    assert B.launches() > 0
    B.close()


def test_batch_single_cell_rows_and_small_problems(nd):
    """Degenerate shapes: 1 x n strips and problems smaller than a tile."""
    import torch
    probs = []
    for (nx, ny) in ((1, 40), (40, 1), (3, 3), (65, 2)):
        d = W.diffusion2d(W.loguniform_alpha(nx, ny, 5 + nx))
        probs.append(dict(n=(nx, ny, 1), diags=d, b=W.uniform_rhs(nx * ny, 9 + ny)))
    B = nd.Batch(probs, tile=32)
    b = torch.tensor(_concat(probs), device="cuda")
    x = torch.zeros_like(b)
    infos = B.solve(b, x, rtol=1e-8)
    xs = x.cpu().numpy()
    for k, p in enumerate(probs):
        assert infos[k]["relres"] <= 1e-8
        assert _true_relres(p, xs[B.offsets[k]:B.offsets[k + 1]]) <= 1e-8
    B.close()
