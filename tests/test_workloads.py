"""The seeded synthetic inputs (paper_1008_3699_gb300/workloads.py): the same
seed gives the same bits, the matrices have the stated structure (zero
entries outside the grid, symmetric diffusion operators, weak diagonal
dominance), and the batch, serving and eikonal recipes have the stated
shapes and ranges."""
import numpy as np
import pytest

from paper_1008_3699_gb300 import workloads as W
from tests.oracle_dense import assemble, full_n, neighbours


def test_same_seed_same_bits():
    a, b = W.varcoef2d_problem(96, 4, 7), W.varcoef2d_problem(96, 4, 7)
    assert np.array_equal(a["diags"], b["diags"]) and np.array_equal(a["b"], b["b"])
    c = W.varcoef2d_problem(96, 4, 8)
    assert not np.array_equal(a["diags"], c["diags"])


@pytest.mark.parametrize("make,n,s", [
    (lambda: W.poisson2d(9, 7), (9, 7, 1), 5),
    (lambda: W.poisson3d(5, 4, 3), (5, 4, 3), 7),
    (lambda: W.diffusion2d(W.smoothed_lognormal_alpha(11, 8, 3)), (11, 8, 1), 5),
    (lambda: W.convdiff9(10, 4.0, 0.7), (10, 10, 1), 9),
])
def test_entries_outside_the_grid_are_zero_and_rows_dominant(make, n, s):
    d = make()
    nb = neighbours(full_n(n), s)
    assert np.all(d[nb < 0] == 0.0)
    assert np.all(d[0] > 0)
    assert np.all(d[0] >= np.abs(d[1:]).sum(axis=0) * (1 - 1e-12))


@pytest.mark.parametrize("make,n,s", [
    (lambda: W.poisson2d(9, 7), (9, 7), 5),
    (lambda: W.diffusion2d(W.loguniform_alpha(8, 6, 5)), (8, 6), 5),
    (lambda: W.poisson3d(4, 5, 3), (4, 5, 3), 7),
])
def test_diffusion_operators_are_symmetric(make, n, s):
    A = assemble(full_n(n), s, make()).toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


def test_batch_and_serving_recipes():
    probs = W.batched_problems(count=20, lo=32, hi=64, seed=9)
    assert len(probs) == 20
    for p in probs:
        nx, ny, _ = p["n"]
        assert 32 <= nx <= 64 and 32 <= ny <= 64
        assert p["diags"].shape == (5, nx * ny) and p["b"].shape == (nx * ny,)
    t, reqs = W.serving_trace(400, rate=2000.0, seed=3)
    assert np.all(np.diff(t) > 0) and 0.1 < t[-1] < 0.3  # 400 arrivals at 2000/s
    kinds = [r["kind"] for r in reqs]
    assert 100 < kinds.count("convdiff9") < 300
    for r in reqs:
        lo, hi = ((64, 2048) if r["kind"] == "convdiff9" else (32, 192))
        assert lo <= r["side"] <= hi


def test_eikonal_recipe_and_embedding():
    p = W.eikonal_problem(64, 4, 1006, sources=4)
    assert p["f"].shape == (64 * 64,) and np.all(p["f"] > 0)
    src = p["sources"]
    assert 1 <= src.size <= 4 and np.all(p["u0"][src] == 0.0)
    assert np.isinf(p["u0"]).sum() == 64 * 64 - src.size
    d9 = W.embed5in9(W.poisson2d(6, 5))
    assert d9.shape == (9, 30) and np.all(d9[5:] == 0.0)
    assert np.array_equal(d9[:5], W.poisson2d(6, 5))
