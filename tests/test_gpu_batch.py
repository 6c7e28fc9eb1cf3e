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
    l0 = B.launches()
    infos = B.solve(b, x, rtol=1e-8)
    # the inner iterations of a refinement step are one graph launch: the
    # launches of a solve do not grow with its iterations
    dl, outer = B.launches() - l0, max(i["outer"] for i in infos)
    assert dl <= 40 * (outer + 1), (dl, outer, max(i["iters"] for i in infos))
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
    l0 = B.launches()
    infos = B.solve(b, x, rtol=1e-8)
    # the inner iterations of a refinement step are one graph launch: the
    # launches of a solve do not grow with its iterations
    dl, outer = B.launches() - l0, max(i["outer"] for i in infos)
    assert dl <= 40 * (outer + 1), (dl, outer, max(i["iters"] for i in infos))
    xs = x.cpu().numpy()
    for k, p in enumerate(probs):
        assert infos[k]["relres"] <= 1e-8
        assert _true_relres(p, xs[B.offsets[k]:B.offsets[k + 1]]) <= 1e-8
    B.close()


@pytest.mark.parametrize("tile", [32, 64, 128])
def test_batched_ssor_apply_matches_the_oracle(nd, tile):
    """One batched SSOR apply (fp32, omega 1.2) of uneven problems against the
    oracle's decomposed SSOR apply (Sec. 5, SPD form) of each problem with the
    same partition, cell by cell, at the fp32 tolerance 2e-5 (unit roundoff
    6e-8 times the growth along a wavefront of a few hundred cells), for every
    tile side the autotuner can choose."""
    import torch
    probs = _problems(9, 20, 300, 91) + W.batched_problems(1, 1, 40, 5)
    om = 1.2
    B = nd.Batch(probs, tile=tile, omega=om)
    r = np.concatenate([W.uniform_rhs(p["n"][0] * p["n"][1], 300 + k) for k, p in enumerate(probs)])
    z = torch.empty(len(r), dtype=torch.float32, device="cuda")
    B.ssor_apply(torch.tensor(r, dtype=torch.float32, device="cuda"), z)
    got = z.cpu().numpy().astype(np.float64)
    off = B.offsets
    for k, p in enumerate(probs):
        nx, ny = int(p["n"][0]), int(p["n"][1])
        sub = (-(-nx // tile), -(-ny // tile), 1)
        ref = oracle.Problem(2, p["n"], 5, p["diags"], sub)
        rk = r[off[k]:off[k + 1]].astype(np.float32).astype(np.float64)  # the fp32 input the GPU saw
        want = ref.ssor_apply(oracle.DECOMPOSED, om, rk)
        err = np.max(np.abs(got[off[k]:off[k + 1]] - want)) / np.max(np.abs(want))
        assert err <= 2e-5, (k, (nx, ny), sub, err)
    B.close()


def test_batched_inner_counts_match_the_oracle(nd):
    """With rtol 1e-3 one refinement step suffices, and its fp32 inner PCG runs
    to ||r|| <= 5e-4 ||b|| (half the outer tolerance, far above fp32 rounding):
    per problem, the count is compared with the oracle's fp64 SSOR-PCG run to
    the same relative residual (SSOR inside CG, Sec. 5). fp32 CG loses
    orthogonality faster than fp64 CG, which delays it by a few percent that
    grow with the count (measured on the GB300: 0 to +12 iterations on counts
    of 87-195), so this is a bounded-lag check: never ahead of the oracle by
    more than 1, behind by at most 10 % (a different preconditioner moves the
    count by far more). The preconditioner itself is pinned cell by cell by the
    apply test above. At tighter outer
    tolerances the fp32 inner solve's true residual stalls near 1e-5 on some
    problems and the refinement takes more steps, so counts are not comparable
    there."""
    import torch
    probs = _problems(8, 24, 200, 19)
    B = nd.Batch(probs, tile=64)
    b = torch.tensor(_concat(probs), device="cuda")
    x = torch.zeros_like(b)
    infos = B.solve(b, x, rtol=1e-3)
    B.close()
    for k, p in enumerate(probs):
        assert infos[k]["outer"] == 1, (k, infos[k])
        nx, ny = int(p["n"][0]), int(p["n"][1])
        sub = (-(-nx // 64), -(-ny // 64), 1)
        ref = oracle.Problem(2, p["n"], 5, p["diags"], sub)
        b32 = p["b"].astype(np.float32).astype(np.float64)
        _, info = ref.solve(oracle.PCG, oracle.PREC_SSOR, oracle.DECOMPOSED, 1.0, 5e-4, 20000, b32)
        slack = max(2, int(np.ceil(0.10 * info["iters"])))
        assert -1 <= infos[k]["iters"] - info["iters"] <= slack, (k, (nx, ny), infos[k]["iters"], info["iters"])
