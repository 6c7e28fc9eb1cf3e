"""Decomposed fast sweeping on the GPU (eikonal_sweep / eikonal_solve) against
the oracle's sweep: every sweep bit-identical (values and the largest change),
whole solves with the same sweep count and bit-identical results, the stop
rule with delta > 0, the degenerate cases, the argument checks, and the
2048^2 workload (16 x 16 subdomains): its first sweep and its whole solve."""
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


def _case(n, seed, sources=3):
    g = np.random.default_rng(seed)
    f = np.exp(0.5 * g.standard_normal(n[0] * n[1]))
    u0 = oracle.eikonal_init(n[0] * n[1], g.integers(0, n[0] * n[1], size=sources))
    return f, u0


CASES = [
    ((64, 48), (2, 2), 1),
    ((131, 97), (3, 4), 2),     # ragged parts
    ((200, 150), (4, 3), 3),
    ((40, 300), (1, 3), 4),     # tall strips
    ((256, 256), (2, 2), 5),    # 128 x 128 subdomains, as in the 2048^2 workload
    ((70, 600), (1, 3), 8),     # 200 rows: seven warps per subdomain
    ((97, 1), (5, 1), 6),       # one row
]


@pytest.mark.parametrize("n,sub,seed", CASES)
def test_sweeps_bit_identical(nd, n, sub, seed):
    import torch
    f, u0 = _case(n, seed)
    h = 1.0 / max(n)
    ref = oracle.Eikonal(n, h, f, sub)
    e = nd.Eikonal(n, h, f, sub)
    a = torch.tensor(u0, device="cuda")
    b = torch.empty_like(a)
    u = u0
    for t in range(9):
        ch = e.sweep(t, a, b)
        u, ch_ref = ref.sweep(t, u)
        np.testing.assert_array_equal(b.cpu().numpy(), u)
        assert ch == ch_ref
        a, b = b, a
    e.close()


@pytest.mark.parametrize("n,sub,seed", CASES[:4])
@pytest.mark.parametrize("delta", [0.0, 1e-6])
def test_solve_matches_oracle(nd, n, sub, seed, delta):
    import torch
    f, u0 = _case(n, seed)
    h = 1.0 / max(n)
    u_ref, info_ref = oracle.Eikonal(n, h, f, sub).solve(u0, delta=delta)
    e = nd.Eikonal(n, h, f, sub)
    u = torch.tensor(u0, device="cuda")
    info = e.solve(u, delta=delta)
    e.close()
    assert info["converged"] and info_ref["converged"]
    assert info["sweeps"] == info_ref["sweeps"]
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_host_vector_and_degenerate_cases(nd):
    # host u, a single cell, no source, zero slowness around a source
    f, u0 = _case((50, 40), 7)
    e = nd.Eikonal((50, 40), 0.02, f, (2, 2))
    u = u0.copy()
    info = e.solve(u)
    u_ref, info_ref = oracle.Eikonal((50, 40), 0.02, f, (2, 2)).solve(u0)
    assert info["sweeps"] == info_ref["sweeps"]
    np.testing.assert_array_equal(u, u_ref)
    e.close()
    one = nd.Eikonal((1, 1), 1.0, np.ones(1), (1, 1))
    u1 = np.zeros(1)
    assert one.solve(u1)["sweeps"] == 4 and u1[0] == 0.0
    one.close()
    none = nd.Eikonal((30, 20), 0.1, np.ones(600), (2, 2))
    u2 = np.full(600, np.inf)
    info2 = none.solve(u2)
    assert info2["sweeps"] == 4 and info2["change"] == 0.0 and np.isinf(u2).all()
    none.close()
    f0 = np.ones(900)
    f0[300:600] = 0.0
    z = nd.Eikonal((30, 30), 0.1, f0, (3, 3))
    u3 = oracle.eikonal_init(900, [450])
    u3_ref, _ = oracle.Eikonal((30, 30), 0.1, f0, (3, 3)).solve(u3)
    z.solve(u3)
    np.testing.assert_array_equal(u3, u3_ref)
    z.close()


def test_refused_arguments(nd):
    import torch
    with pytest.raises(nd.NdiagError):
        nd.Eikonal((16, 16), 0.0, np.ones(256))
    with pytest.raises(nd.NdiagError):
        nd.Eikonal((16, 16), 1.0, -np.ones(256))
    bad = np.ones(256)
    bad[3] = np.nan
    with pytest.raises(nd.NdiagError):
        nd.Eikonal((16, 16), 1.0, bad)
    with pytest.raises(nd.NdiagError):
        nd.Eikonal((16, 16), 1.0, np.ones(256), (17, 1))
    with pytest.raises(nd.NdiagError):
        nd.Eikonal((40, 400), 1.0, np.ones(16000), (1, 1))  # more than 256 rows
    e = nd.Eikonal((16, 16), 1.0, np.ones(256), (2, 2))
    a = torch.zeros(256, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdiagError):
        e.sweep(0, a, a)
    e.close()


def test_full_size_workload(nd):
    import torch
    p = W.eikonal_problem()
    ref = oracle.Eikonal(p["n"], p["h"], p["f"], p["sub"])
    e = nd.Eikonal(p["n"], p["h"], p["f"], p["sub"])
    a = torch.tensor(p["u0"], device="cuda")
    b = torch.empty_like(a)
    ch = e.sweep(0, a, b)
    u1, ch_ref = ref.sweep(0, p["u0"])
    np.testing.assert_array_equal(b.cpu().numpy(), u1)
    assert ch == ch_ref
    u_ref, info_ref = ref.solve(p["u0"])
    info = e.solve(a)
    e.close()
    assert info["converged"] and info["sweeps"] == info_ref["sweeps"]
    np.testing.assert_array_equal(a.cpu().numpy(), u_ref)
