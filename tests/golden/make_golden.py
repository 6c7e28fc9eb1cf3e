"""Write stored expected values for the full-size workloads by running the CPU
oracle (oracle/) on the seeded inputs (paper_1008_3699_gb300/workloads.py).

Nothing here touches the CUDA library. Usage:
    python tests/golden/make_golden.py poisson64   # seconds
    python tests/golden/make_golden.py varcoef2048 # long: two full 2048^2 solves
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


JOBS = {"poisson64": poisson64, "varcoef2048": varcoef2048}

if __name__ == "__main__":
    oracle.build()
    for name in sys.argv[1:]:
        res = JOBS[name]()
        res["_source"] = "written by tests/golden/make_golden.py from the CPU oracle"
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(res, f, indent=1)
        print(name, res)
