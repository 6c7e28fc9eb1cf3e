"""The oracle's per-iteration Krylov record (the reference of the GPU lockstep
tests) pinned to independent computations: scipy's BiCGSTAB and CG iterates
with the same preconditioner, and the first BiCGSTAB iteration written out from
its definition (van der Vorst 1992) with scipy's sparse product."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_1008_3699_gb300 import workloads as W
from tests.test_oracle_pins import _random_diags, assemble

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _setup(orc, kind):
    n, N = (20, 17, 1), 340
    b = W.uniform_rhs(N, 4)
    if kind == "bicgstab":
        d = _random_diags(n, 5, 21)
        pb = orc.Problem(2, n, 5, d, (2, 3))
        pb.ilu0_factor(orc.DECOMPOSED)
        M = lambda r: pb.ilu0_apply(r)
    else:
        d = W.diffusion2d(W.loguniform_alpha(20, 17, 3))
        pb = orc.Problem(2, n, 5, d, (2, 3))
        M = lambda r: pb.ssor_apply(orc.DECOMPOSED, 1.0, r)
    return n, N, b, d, pb, M


@pytest.mark.parametrize("kind", ["bicgstab", "pcg"])
def test_recorded_residuals_follow_scipy_iterates(orc, kind):
    """||r_k|| / ||b|| of the record against the true residual of scipy's k-th
    iterate (the recurrence and the true residual agree to rounding while both
    are far above it)."""
    n, N, b, d, pb, M = _setup(orc, kind)
    A = assemble(n, 5, d).tocsr()
    if kind == "bicgstab":
        _, info = pb.solve(orc.BICGSTAB, orc.PREC_ILU0, orc.DECOMPOSED, 1.0, 1e-10, 300, b)
        col, solver = 1, spla.bicgstab
    else:
        _, info = pb.solve(orc.PCG, orc.PREC_SSOR, orc.DECOMPOSED, 1.0, 1e-10, 300, b)
        col, solver = 0, spla.cg
    true_rel = []
    solver(A, b, rtol=1e-10, atol=0, M=spla.LinearOperator((N, N), matvec=M), maxiter=12,
           callback=lambda xk: true_rel.append(np.linalg.norm(b - A @ xk) / np.linalg.norm(b)))
    rec = info["history"][:, col]
    k = min(10, len(true_rel))
    assert k >= 8
    assert np.allclose(rec[:k], true_rel[:k], rtol=1e-7, atol=1e-13), (rec[:k], true_rel[:k])
    assert info["history"].shape == (info["iters"], 4)


def test_first_bicgstab_iteration_from_its_definition(orc):
    """x0 = 0: r0 = b, r^ = r0, p = r0; alpha = (r^, r0) / (r^, A M p);
    s = r0 - alpha A M p; omega = (t, s) / (t, t) with t = A M s; r1 = s - omega t."""
    n, N, b, d, pb, M = _setup(orc, "bicgstab")
    A = assemble(n, 5, d).tocsr()
    _, info = pb.solve(orc.BICGSTAB, orc.PREC_ILU0, orc.DECOMPOSED, 1.0, 1e-10, 300, b)
    r0 = b.copy()
    v = A @ M(r0)
    alpha = (r0 @ r0) / (r0 @ v)
    s = r0 - alpha * v
    t = A @ M(s)
    omega = (t @ s) / (t @ t)
    r1 = s - omega * t
    bn = np.linalg.norm(b)
    want = [np.linalg.norm(s) / bn, np.linalg.norm(r1) / bn, alpha, omega]
    assert np.allclose(info["history"][0], want, rtol=1e-12, atol=0), (info["history"][0], want)


def test_stored_full_size_record_is_self_consistent():
    """The stored 2048^2 record: 40 rows of four finite values, ||r|| <= ||s||
    in the early rows (omega minimises ||s - omega t||), a spread that starts at
    rounding level and grows, and decomposed and natural records that differ
    (different preconditioners) well beyond that spread."""
    g = json.load(open(os.path.join(HERE, "golden", "varcoef2048_history.json")))
    for name in ("decomposed", "natural"):
        h, dev = np.array(g[name]["history"]), np.array(g[name]["dev"])
        assert h.shape == (40, 4) and np.all(np.isfinite(h))
        assert np.all(h[:20, 1] <= h[:20, 0] * (1 + 1e-12))
        assert dev[0] < 1e-13 and dev[20] > 100 * dev[0]
    a, b = np.array(g["decomposed"]["history"]), np.array(g["natural"]["history"])
    assert np.max(np.abs(a[0] - b[0]) / np.abs(b[0])) > 1e6 * g["decomposed"]["dev"][0]
