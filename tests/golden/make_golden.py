"""Write stored expected values for the full-size workloads by running the CPU
oracle (oracle/) on the seeded inputs (paper_1008_3699_gb300/workloads.py).

Nothing here touches the CUDA library. Usage:
    python tests/golden/make_golden.py poisson64   # seconds
    python tests/golden/make_golden.py varcoef2048 # long: two full 2048^2 solves
    python tests/golden/make_golden.py varcoef2048_envelope  # long: 7 perturbed solves in parallel
    python tests/golden/make_golden.py varcoef2048_mg  # long: one 2048^2 multigrid-PCG solve
    python tests/golden/make_golden.py poisson3d256_mg  # long: one 256^3 multigrid-PCG solve (about 10 GB)
    python tests/golden/make_golden.py varcoef2048_history  # minutes: 40 BiCGSTAB iterations, 5 b's, 2 orders
Output: tests/golden/<name>.json
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1008_3699_gb300 import workloads as W  # noqa: E402


def poisson64():
    p = W.poisson64_problem()
    out = {}
    for name, mode in (("natural", oracle.NATURAL), ("decomposed", oracle.DECOMPOSED)):
        pb = oracle.Problem(2, p["n"], 5, p["diags"], p["sub"] if mode else (1, 1))
        t0 = time.time()
        x, info = pb.solve(oracle.STATIONARY, oracle.PREC_NONE, mode, p["omega"], 1e-8, 100000, p["b"])
        out[name] = dict(iters=info["iters"], relres=info["relres"], seconds=time.time() - t0,
                         x_norm=float(np.linalg.norm(x)))
    return out


def varcoef2048(n=2048, sub=16):
    p = W.varcoef2d_problem(n, sub)
    out = {}
    for name, mode in (("decomposed", oracle.DECOMPOSED), ("natural", oracle.NATURAL)):
        pb = oracle.Problem(2, p["n"], 5, p["diags"], p["sub"] if mode else (1, 1))
        t0 = time.time()
        pb.ilu0_factor(mode)
        x, info = pb.solve(oracle.BICGSTAB, oracle.PREC_ILU0, mode, 1.0, 1e-8, 20000, p["b"])
        out[name] = dict(iters=info["iters"], relres=info["relres"], seconds=time.time() - t0,
                         x_norm=float(np.linalg.norm(x)))
        print(name, out[name], flush=True)
    return out


def varcoef2048_mg(n=2048, sub=16, omega=0.9):
    """Oracle multigrid-PCG (oracle/mg.py) on the 2048^2 workload."""
    import oracle.mg as mg
    p = W.varcoef2d_problem(n, sub)
    t0 = time.time()
    H = mg.Hierarchy(n, n, p["diags"], p["sub"], omega)
    x, info = mg.pcg(H, p["b"], 1e-8, 2000)
    out = dict(omega=omega, levels=len(H.levels), iters=info["iters"], relres=info["relres"],
               status=info["status"], seconds=time.time() - t0, x_norm=float(np.linalg.norm(x)))
    print(out, flush=True)
    return out


def poisson3d256_mg(n=256, sub=8, omega=0.9):
    """Oracle 3D multigrid-PCG (oracle/mg.py) on the 256^3 Poisson workload."""
    import oracle.mg as mg
    p = W.poisson3d_problem(n, sub)
    t0 = time.time()
    H = mg.Hierarchy3(p["n"], p["diags"], p["sub"], omega)
    x, info = mg.pcg(H, p["b"], 1e-8, 500)
    out = dict(omega=omega, levels=len(H.levels), iters=info["iters"], relres=info["relres"],
               status=info["status"], seconds=time.time() - t0, x_norm=float(np.linalg.norm(x)))
    print(out, flush=True)
    return out


def _perturbed_solve(k, n=2048, sub=16):
    """Oracle BiCGSTAB count of the 2048^2 workload with b scaled by
    (1 + 1e-15 g), g ~ N(0, 1) from seed 4242 + k (rounding-level change)."""
    import oracle as orc
    p = W.varcoef2d_problem(n, sub)
    g = np.random.default_rng(4242 + k)
    b = p["b"] * (1.0 + 1e-15 * g.standard_normal(p["b"].shape[0]))
    pb = orc.Problem(2, p["n"], 5, p["diags"], p["sub"])
    pb.ilu0_factor(orc.DECOMPOSED)
    _, info = pb.solve(orc.BICGSTAB, orc.PREC_ILU0, orc.DECOMPOSED, 1.0, 1e-8, 20000, b)
    return dict(k=k, iters=info["iters"], relres=info["relres"])


def varcoef2048_envelope(count=7):
    """Spread of the oracle's decomposed BiCGSTAB count under 1e-15 relative
    perturbations of b (one process per solve, spawned)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(count) as pool:
        runs = pool.map(_perturbed_solve, range(count))
    its = [r["iters"] for r in runs]
    return dict(perturbation="b * (1 + 1e-15 g), g ~ N(0,1), seeds 4242..", runs=runs, min=min(its), max=max(its))


HIST_ITERS, HIST_SEEDS = 40, 4


def _history_run(args):
    """First HIST_ITERS rows of the oracle's BiCGSTAB + ILU(0) record on the
    2048^2 workload (mode: 1 decomposed 16 x 16, 0 natural), with b scaled by
    (1 + 1e-15 g), g ~ N(0, 1) from seed 5151 + k, or unperturbed for k < 0."""
    mode, k, n, sub = args
    import oracle as orc
    p = W.varcoef2d_problem(n, sub)
    b = p["b"]
    if k >= 0:
        g = np.random.default_rng(5151 + k)
        b = b * (1.0 + 1e-15 * g.standard_normal(b.shape[0]))
    pb = orc.Problem(2, p["n"], 5, p["diags"], p["sub"] if mode else (1, 1))
    pb.ilu0_factor(mode)
    _, info = pb.solve(orc.BICGSTAB, orc.PREC_ILU0, mode, 1.0, 1e-8, HIST_ITERS, b)
    return mode, k, info["history"].tolist()


def varcoef2048_history(n=2048, sub=16):
    """The oracle's BiCGSTAB + ILU(0) iteration record (||s||/||b||, ||r||/||b||,
    alpha, omega) over the first HIST_ITERS iterations, decomposed and natural,
    and its own spread under rounding-level changes of b: dev[k] = the largest
    relative change of any of the four values at iteration k over HIST_SEEDS
    perturbed right-hand sides (one process per solve, spawned)."""
    import multiprocessing as mp
    jobs = [(m, k, n, sub) for m in (1, 0) for k in range(-1, HIST_SEEDS)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        runs = pool.map(_history_run, jobs)
    out = dict(iters=HIST_ITERS, seeds=HIST_SEEDS, perturbation="b * (1 + 1e-15 g), g ~ N(0,1), seeds 5151..")
    for m, name in ((1, "decomposed"), (0, "natural")):
        base = np.array(next(h for mm, k, h in runs if mm == m and k < 0))
        dev = np.zeros(len(base))
        for mm, k, h in runs:
            if mm != m or k < 0:
                continue
            h = np.array(h)
            r = min(len(h), len(base))
            dev[:r] = np.maximum(dev[:r], np.max(np.abs(h[:r] - base[:r]) / np.abs(base[:r]), axis=1))
        out[name] = dict(history=base.tolist(), dev=dev.tolist())
    return out


JOBS = {"poisson64": poisson64, "varcoef2048": varcoef2048, "varcoef2048_envelope": varcoef2048_envelope,
        "varcoef2048_mg": varcoef2048_mg, "poisson3d256_mg": poisson3d256_mg,
        "varcoef2048_history": varcoef2048_history}

if __name__ == "__main__":
    oracle.build()
    for name in sys.argv[1:]:
        res = JOBS[name]()
        res["_source"] = "written by tests/golden/make_golden.py from the CPU oracle"
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(res, f, indent=1)
        print(name, res)
