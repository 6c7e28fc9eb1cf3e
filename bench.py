#!/usr/bin/env python3
"""Benchmark of the decomposed sequential sweep on one GB300.

Workload: 2D variable-coefficient diffusion, 5-point, 2048 x 2048 cells,
alpha = box5x5(exp(N(0,1))) (seeded), b ~ U[-1,1], fp64; the paper's decomposed
ILU(0) over 16 x 16 subdomains as the preconditioner of BiCGSTAB, solved to
||b - A x|| / ||b|| <= 1e-8 from x = 0. One step = ilu0_factor + krylov_solve.

Metric: Gcell-updates/s (cell updates of every sweep kernel in the step: the
factor sweep and the two sweeps of every ILU(0) apply, N cells each, over the
wall time of the whole step), with solves/s and p50/p99 solve latency beside
it, and the roofline of the sweep kernel (algorithmic bytes / device time of
its launches, from CUDA events on the handle's stream).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own copy (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE, SUB = 2048, 16
WORKLOAD = "varcoef2d-2048x2048-5pt-fp64-ilu0-bicgstab-16x16"
METRIC = "Gcell-updates/s per sweep (% HBM peak); solves/s and p99 latency at rel-res 1e-8"
SWEEP_SRC = os.path.join(ROOT, "paper_1008_3699_gb300", "csrc", "sweep2d_staged.cu")
PROFILE = os.path.join(ROOT, "profiles", "sweep2d_staged_ilu0_varcoef2048.md")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic():
    """dram bytes per launch of the sweep kernel from the committed ncu summary,
    only if the kernel source is unchanged since the counters were taken."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m or not t:
        return None
    sha = hashlib.sha256(open(SWEEP_SRC, "rb").read()).hexdigest()
    return float(t.group(1)) if sha == m.group(1) else None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(problem, iters=6):
    """The oracle as it stands, on one host core: the ILU(0) factor and a bounded
    number of BiCGSTAB iterations of the same workload."""
    import oracle
    oracle.build()
    pb = oracle.Problem(2, problem["n"], 5, problem["diags"], problem["sub"])
    t0 = time.perf_counter()
    pb.ilu0_factor(oracle.DECOMPOSED)
    _, info = pb.solve(oracle.BICGSTAB, oracle.PREC_ILU0, oracle.DECOMPOSED, 1.0, 1e-8, iters, problem["b"])
    dt = time.perf_counter() - t0
    N = problem["n"][0] * problem["n"][1]
    sweeps = 1 + 4 * info["iters"]  # factor + two applies (two sweeps each) per iteration
    return {"value": N * sweeps / dt / 1e9, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"ILU(0) factor + {info['iters']} BiCGSTAB iterations of the 2048^2 workload "
                      f"({sweeps} sweeps, {dt:.1f} s, 1 thread)", "seconds": dt}


def over_ranks(ms, updates, dist, device):
    """Whole-job timing of replicas: the slowest rank's time and the cell
    updates of all ranks (dist = torch.distributed or None)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1008_3699_gb300 import workloads as W
    problem = W.varcoef2d_problem(N_SIDE, SUB)
    vals = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(problem, iters=2)
        if k >= args.warmup:
            vals.append(r)
    v = statistics.median(x["value"] for x in vals)
    N = N_SIDE * N_SIDE
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gcell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_SIDE, N_SIDE], "subdomains": [SUB, SUB]},
        "cpu_baseline": {"value": v, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # one step = the bounded sample above (factor + 2 iterations), timed on the host
        "ms_per_step": 1e3 * statistics.median(x["seconds"] for x in vals),
    }))


def progress(msg):
    """Where the run is, on stderr (the JSON line is the only stdout output)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-natural", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--kernel-only", type=int, default=0, metavar="K",
                    help="only factor and run K ILU(0) applies of the workload (for kernel profiling)")
    ap.add_argument("--workload", default="varcoef2048",
                    choices=["varcoef2048", "poisson64", "poisson3d", "batch512", "serving", "mg2048",
                             "eikonal2048", "mg3d", "convdiff9"],
                    help="varcoef2048 is the benchmark; the others print one measurement line each")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--n3d", type=int, default=256, help="side of the 3D Poisson workload (subdomains of 32^3)")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the 256^3 fp32 + refinement and 512-problem batch sub-measurements")
    ap.add_argument("--roofline-iters", type=int, default=200,
                    help="BiCGSTAB iterations of the pass that times every sweep launch")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "varcoef2048":
        return EXTRA[args.workload](args)

    import numpy as np
    import torch
    from paper_1008_3699_gb300 import build as nd_build
    from paper_1008_3699_gb300 import ndiag as nd
    from paper_1008_3699_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and "RANK" in os.environ:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    nd_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()

    problem = W.varcoef2d_problem(N_SIDE, SUB)
    N = N_SIDE * N_SIDE
    if args.kernel_only:
        h = nd.NDiag(2, problem["n"], 5, problem["diags"], problem["sub"], "fp64")
        h.ilu0_factor(nd.DECOMPOSED)
        r = torch.tensor(problem["b"], device="cuda")
        z = torch.empty_like(r)
        for _ in range(args.kernel_only):
            h.ilu0_apply(r, z)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": args.kernel_only, "z_norm": float(z.norm())}))
        return
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        progress("oracle sample on the host")
        cpu = cpu_baseline(problem)  # host only, before the GPU work
    progress("warm-up steps")

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = nd.NDiag(2, problem["n"], 5, problem["diags"], problem["sub"], "fp64", stream=stream)
        b = torch.tensor(problem["b"], device="cuda")
        x = torch.zeros(N, dtype=torch.float64, device="cuda")

        def step():
            h.ilu0_factor(nd.DECOMPOSED)
            x.zero_()
            return h.solve(nd.BICGSTAB, nd.PREC_ILU0, b, x, rtol=1e-8, maxit=20000)

        for _ in range(args.warmup):
            info = step()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        progress("timed steps")
        clocks = Clocks(uuid)
        barrier()
        torch.cuda.synchronize()
        h.profile(False)  # counters only: the iteration runs as captured graphs
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        infos = []
        for k in range(args.steps):
            infos.append(step())
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        cnt = h.counters()
        lat = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        total_ms, all_updates = over_ranks(ev[0].elapsed_time(ev[-1]), float(N) * cnt["sweep_launches"], dist,
                                           "cuda")
        value = all_updates / (total_ms / 1e3) / 1e9

        progress("roofline pass")
        # roofline pass: a bounded solve of the same system with every sweep
        # launch timed by CUDA events on the handle's stream (the iteration is
        # then launched kernel by kernel, not as graphs)
        h.profile(True)
        x.zero_()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        h.solve(nd.BICGSTAB, nd.PREC_ILU0, b, x, rtol=1e-8, maxit=args.roofline_iters, raise_on_noconv=False)
        r1.record(stream)
        torch.cuda.synchronize()
        pc = h.counters()
        pass_ms = r0.elapsed_time(r1)
        h.profile(False)

        progress("end-to-end steps")
        # end to end through the C ABI with pinned host buffers
        hb = torch.empty(N, dtype=torch.float64, pin_memory=True)
        hb.copy_(torch.from_numpy(problem["b"]))
        hx = torch.empty(N, dtype=torch.float64, pin_memory=True)
        hd = torch.empty(problem["diags"].shape, dtype=torch.float64, pin_memory=True)
        hd.copy_(torch.from_numpy(problem["diags"]))
        hb_np, hx_np, hd_np = hb.numpy(), hx.numpy(), hd.numpy()
        e2e_updates, e2e_s = 0.0, 0.0
        for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = nd.NDiag(2, problem["n"], 5, hd_np, problem["sub"], "fp64", stream=stream)
            g.profile(False)
            g.ilu0_factor(nd.DECOMPOSED)
            hx_np[:] = 0.0
            g.solve(nd.BICGSTAB, nd.PREC_ILU0, hb_np, hx_np, rtol=1e-8, maxit=20000)
            c2 = g.counters()
            g.close()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k > 0:  # first one warms the allocator
                e2e_updates += float(N) * c2["sweep_launches"]
                e2e_s += dt
        e2e_val = torch.tensor([e2e_updates / e2e_s / 1e9 * world if e2e_s > 0 else 0.0],
                               dtype=torch.float64, device="cuda")

        natural = None
        if not args.no_natural and rank == 0:
            progress("natural-order comparison")
            hn = nd.NDiag(2, problem["n"], 5, problem["diags"], (1, 1), "fp64", stream=stream)
            hn.ilu0_factor(nd.NATURAL)
            xn = torch.zeros(N, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ni = hn.solve(nd.BICGSTAB, nd.PREC_ILU0, b, xn, rtol=1e-8, maxit=20000, mode=nd.NATURAL,
                          raise_on_noconv=False)
            torch.cuda.synchronize()
            natural = {"iters": ni["iters"], "relres": ni["relres"], "seconds": time.perf_counter() - t0}
            hn.close()

        extras = None
        if not args.no_extras and rank == 0:
            progress("256^3 fp32 + refinement")
            e3 = extra_fp32_refine_3d(torch, nd, W, args, 256)
            progress("512-problem batch")
            extras = {"fp32_refine_256cube": e3, "batch512": extra_batch512(torch, nd, W, args)}

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    # algorithmic bytes of an fp64 ILU(0) apply: 80 B a cell (forward: two L
    # entries, the pivot, r, y; backward: two U entries, the pivot, y, z), i.e.
    # 40 B a cell for each of its two sweeps; the kernels' own count is 32 B (the
    # unit form; the pivot scaling is read by the vector kernels instead)
    B8D = 40.0
    sweep_s = pc["sweep_ms"] / 1e3
    achieved = B8D * N * pc["sweep_launches"] / sweep_s / 1e9 if sweep_s > 0 else None
    achieved_kernel = pc["sweep_bytes"] / sweep_s / 1e9 if sweep_s > 0 else None
    lat_sorted = sorted(lat)
    p = lambda q: lat_sorted[min(len(lat_sorted) - 1, int(round(q * (len(lat_sorted) - 1))))]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Gcell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_SIDE, N_SIDE], "subdomains": [SUB, SUB],
                   "method": "BiCGSTAB + decomposed ILU(0)", "rtol": 1e-8, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (matrix 168 MB + 9 vectors of 34 MB vs 129 MB L2)"},
        "solves_per_s": world * args.steps / (total_ms / 1e3),
        "latency_ms": {"p50": p(0.5), "p99": p(0.99)},
        "iters": [i["iters"] for i in infos],
        "relres": max(i["relres"] for i in infos),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": kernel_traffic(),
                     "bytes_per_cell": B8D,
                     "bytes_basis": "algorithmic bytes of an fp64 ILU(0) apply, 80 B a cell = 2 sweeps x 40",
                     "kernel": "sweep2d_staged_kernel (the two sweeps of every ILU(0) apply)",
                     "peak_kind": peak_kind, "sweep_launches": pc["sweep_launches"], "sweep_ms": pc["sweep_ms"],
                     "avg_launch_us": 1e3 * pc["sweep_ms"] / pc["sweep_launches"] if pc["sweep_launches"] else None,
                     "timed_pass": f"{args.roofline_iters} BiCGSTAB iterations of the same system, "
                                   "every sweep launch bracketed by CUDA events on the handle's stream",
                     "kernel_counted": {"bytes_per_cell": 32.0, "achieved": achieved_kernel,
                                        "frac": (achieved_kernel / peak) if achieved_kernel else None}},
        "sweep_share_of_step": pc["sweep_ms"] / pass_ms if pass_ms else None,
        "gpu_launches": cnt["launches"],
        "e2e": {"value": float(e2e_val.item()), "unit": "Gcell-updates/s",
                "h2d_bytes_per_step": int(hd_np.nbytes + hb_np.nbytes + hx_np.nbytes),
                "d2h_bytes_per_step": int(hx_np.nbytes)},
        "clocks": clk,
        "cpu_baseline": cpu,
        "natural_ilu0": natural,
    }
    if extras:
        line.update(extras)
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Sub-measurements carried in the benchmark line: the 256^3 fp32 + refinement
# solve and the 512-problem batch.
# ---------------------------------------------------------------------------

def extra_fp32_refine_3d(torch, nd, W, args, n):
    """n^3 Poisson, 32^3 subdomains: fp32 SSOR-PCG with fp64 residuals and
    refinement to rel-res 1e-8 (one warm-up solve, one timed), the fp32 SSOR
    apply timed with CUDA events, and the oracle's fp64 SSOR apply on a 128^3
    sample of the same problem family on one host core."""
    p = W.poisson3d_problem(n, max(1, n // 32))
    N = n ** 3
    h = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], "fp32")
    b = torch.tensor(p["b"], device="cuda")
    for _ in range(2):
        x = torch.zeros_like(b)
        info = _timed_solve(torch, h, nd.PCG, nd.PREC_SSOR, b, x, rtol=1e-8, maxit=5000)
    r = b.float()
    z = torch.empty_like(r)
    for _ in range(2):
        h.ssor_apply(1.0, r, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        h.ssor_apply(1.0, r, z)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 5
    h.close()
    # algorithmic bytes of an fp32 7-point SSOR apply: forward (pivot, 3
    # entries, r, tmp) and transposed solve (3 entries, tmp, z), 4 B each
    bpc = 4.0 * ((4 + 2) + (3 + 2))
    peak, kind = measured_peaks()
    gbs = bpc * N / (apply_ms / 1e3) / 1e9
    out = {"workload": f"poisson3d-{n}^3-7pt-fp32-ssor-pcg+fp64-refinement-{max(1, n // 32)}^3",
           "seconds": info["wall_s"], "solves_per_s": 1.0 / info["wall_s"], "iters": info["iters"],
           "outer": info["outer"], "relres": info["relres"], "ssor_apply_ms": apply_ms,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "bytes_per_cell": bpc, "peak_kind": kind,
                        "kernel": "fp32 SSOR apply (sweep3d_kernel block passes + sweep3d_wave_kernel walks)"}}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ns = 128
        q = W.poisson3d_problem(ns, ns // 32)
        pb = oracle.Problem(3, q["n"], 7, q["diags"], q["sub"])
        pb.ssor_apply(oracle.DECOMPOSED, 1.0, q["b"])  # builds the sweep plan
        t0 = time.perf_counter()
        pb.ssor_apply(oracle.DECOMPOSED, 1.0, q["b"])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 2 * ns ** 3 / dt / 1e9, "unit": "Gcell-updates/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"one fp64 SSOR apply (two sweeps) of the oracle at {ns}^3, 32^3 "
                                         f"subdomains ({dt:.2f} s)"}
    return out


def extra_batch512(torch, nd, W, args):
    """512 problems (sides U[32,512], log-uniform coefficients): the batched
    fp32 + fp64-refinement SSOR-PCG (autotuned tile, graph-captured chunks),
    beside fp64 SSOR-PCG with one handle per problem on the first 64 problems,
    and the oracle on the first 4 problems (one host core)."""
    import numpy as np
    probs = W.batched_problems(512, 32, 512, 1004)
    b = torch.tensor(np.concatenate([q["b"] for q in probs]), device="cuda")
    B = nd.Batch(probs, tile=64)
    B.autotune(b)
    for _ in range(2):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = B.solve(b, x, rtol=1e-8)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    out = {"workload": "batch-512x2d-5pt-U[32,512]-fp32+fp64ref-ssor-pcg", "solves_per_s": len(probs) / dt,
           "seconds": dt, "tile": int(B.tiles()[0]), "relres_max": max(i["relres"] for i in infos),
           "iters_mean": float(np.mean([i["iters"] for i in infos])), "launches": B.launches()}
    B.close()
    tot = 0.0
    for q in probs[:64]:
        sub = (max(1, -(-q["n"][0] // 64)), max(1, -(-q["n"][1] // 64)))
        h = nd.NDiag(2, q["n"], 5, q["diags"], sub, "fp64")
        bk = torch.tensor(q["b"], device="cuda")
        tot += _timed_solve(torch, h, nd.PCG, nd.PREC_SSOR, bk, torch.zeros_like(bk), rtol=1e-8,
                            maxit=20000)["wall_s"]
        h.close()
    out["fp64_one_per_handle"] = {"solves_per_s": 64 / tot, "sample": "the first 64 problems, one solve each"}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        for q in probs[:4]:
            sub = (max(1, -(-q["n"][0] // 64)), max(1, -(-q["n"][1] // 64)))
            pb = oracle.Problem(2, q["n"], 5, q["diags"], sub)
            pb.solve(oracle.PCG, oracle.PREC_SSOR, oracle.DECOMPOSED, 1.0, 1e-8, 20000, q["b"])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 4 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                               "sample": f"fp64 SSOR-PCG of the first 4 problems ({dt:.1f} s)"}
    return out


# ---------------------------------------------------------------------------
# The other workloads: one JSON measurement line each (not the benchmark line).
# ---------------------------------------------------------------------------

def _setup():
    import torch
    from paper_1008_3699_gb300 import build as nd_build
    from paper_1008_3699_gb300 import ndiag as nd
    from paper_1008_3699_gb300 import workloads as W
    nd_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    return torch, nd, W


def _timed_solve(torch, h, *a, **kw):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = h.solve(*a, **kw)
    torch.cuda.synchronize()
    info["wall_s"] = time.perf_counter() - t0
    return info


def workload_poisson64(args):
    """64 x 64 Poisson, 2 x 2 subdomains: decomposed and natural-order SOR as
    stationary solvers to rel-res 1e-8 with omega = 2/(1+sin(pi/65))."""
    torch, nd, W = _setup()
    p = W.poisson64_problem()
    out = {}
    for name, mode, sub in (("decomposed", nd.DECOMPOSED, p["sub"]), ("natural", nd.NATURAL, (1, 1, 1))):
        h = nd.NDiag(2, p["n"], 5, p["diags"], sub, "fp64")
        b = torch.tensor(p["b"], device="cuda")
        for k in range(args.warmup + 1):
            x = torch.zeros_like(b)
            info = _timed_solve(torch, h, nd.STATIONARY, nd.PREC_NONE, b, x, rtol=1e-8, maxit=20000,
                                omega=p["omega"], mode=mode)
        out[name] = {k: info[k] for k in ("iters", "relres", "wall_s")}
        h.close()
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    b = torch.tensor(p["b"], device="cuda")
    t0 = time.perf_counter()
    om, its = h.tune_omega(b, rtol=1e-8, maxit=20000, budget=60, omega=p["omega"])
    out["decomposed_tuned_omega"] = {"iters": its, "omega": om, "tune_s": time.perf_counter() - t0}
    h.close()
    print(json.dumps({"workload": "poisson2d-64x64-5pt-fp64-sor-2x2", "metric": "SOR sweeps to rel-res 1e-8",
                      "omega": p["omega"], **out}))


def workload_poisson3d(args):
    """n^3 Poisson (default 256^3), subdomains of 32^3: SSOR-PCG with fp32
    sweeps and fp64 refinement, and the same in fp64, to rel-res 1e-8; SSOR
    apply time (CUDA events around the whole apply)."""
    torch, nd, W = _setup()
    n = args.n3d
    p = W.poisson3d_problem(n, max(1, n // 32))
    N = n ** 3
    out = {}
    for prec in ("fp32", "fp64"):
        h = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], prec)
        dt = torch.float64 if prec == "fp64" else torch.float32
        r = torch.tensor(p["b"], device="cuda", dtype=dt)
        z = torch.empty_like(r)
        for _ in range(max(2, args.warmup)):
            h.ssor_apply(1.0, r, z)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(5):
            h.ssor_apply(1.0, r, z)
        ev1.record()
        torch.cuda.synchronize()
        apply_ms = ev0.elapsed_time(ev1) / 5
        b = torch.tensor(p["b"], device="cuda")
        x = torch.zeros_like(b)
        info = _timed_solve(torch, h, nd.PCG, nd.PREC_SSOR, b, x, rtol=1e-8, maxit=5000)
        # algorithmic bytes of one SSOR apply: forward sweep (inv, 3 entries, r,
        # tmp) and transposed solve (3 entries, tmp, z), each value once
        wc, wv = (8, 8) if prec == "fp64" else (4, 4)
        apply_bytes = N * ((4 * wc + 2 * wv) + (3 * wc + 2 * wv))
        peak, kind = measured_peaks()
        gbs = apply_bytes / (apply_ms / 1e3) / 1e9
        out[prec + "_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                   "frac": gbs / peak, "peak_kind": kind,
                                   "kernel": "SSOR apply (sweep3d_kernel block passes + sweep3d_wave_kernel walks)"}
        out[prec] = {"ssor_apply_ms": apply_ms, "sweep_gcell_per_s": 2 * N / apply_ms / 1e6,
                     **{k: info[k] for k in ("iters", "outer", "relres", "wall_s")}}
        h.close()
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pb = oracle.Problem(3, p["n"], 7, p["diags"], p["sub"])
        pb.ssor_apply(oracle.DECOMPOSED, 1.0, p["b"])  # builds the sweep plan
        t0 = time.perf_counter()
        pb.ssor_apply(oracle.DECOMPOSED, 1.0, p["b"])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 2 * N / dt / 1e9, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                               "sample": f"one fp64 SSOR apply (two sweeps) of the oracle at {n}^3 ({dt:.1f} s)"}
    print(json.dumps({"workload": f"poisson3d-{n}^3-7pt-ssor-pcg-{max(1, n // 32)}^3", "metric": "solve seconds to rel-res 1e-8",
                      **out}))


def workload_batch512(args):
    """512 variable-coefficient 5-point problems (sides U[32,512]): the batched
    fp32 + fp64-refinement SSOR-PCG (autotuned tile, graph-captured chunks)
    against plain fp64 solves of one problem per handle."""
    torch, nd, W = _setup()
    import numpy as np
    probs = W.batched_problems(512, 32, 512, 1004)
    b = torch.tensor(np.concatenate([q["b"] for q in probs]), device="cuda")
    B = nd.Batch(probs, tile=64)
    B.autotune(b)
    for k in range(2):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = B.solve(b, x, rtol=1e-8)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    line = {"workload": "batch-512x2d-5pt-U[32,512]-fp32+fp64ref-ssor-pcg", "metric": "solves/s at rel-res 1e-8",
            "batched": {"solves_per_s": len(probs) / dt, "seconds": dt, "tile": int(B.tiles()[0]),
                        "relres_max": max(i["relres"] for i in infos),
                        "iters_mean": float(np.mean([i["iters"] for i in infos])), "launches": B.launches()}}
    B.close()
    tot, its = 0.0, []
    for q in probs:
        sub = (max(1, -(-q["n"][0] // 64)), max(1, -(-q["n"][1] // 64)))
        h = nd.NDiag(2, q["n"], 5, q["diags"], sub, "fp64")
        bk = torch.tensor(q["b"], device="cuda")
        info = _timed_solve(torch, h, nd.PCG, nd.PREC_SSOR, bk, torch.zeros_like(bk), rtol=1e-8, maxit=20000)
        tot += info["wall_s"]
        its.append(info["iters"])
        h.close()
    line["fp64_one_per_handle"] = {"solves_per_s": len(probs) / tot, "seconds": tot,
                                   "iters_mean": float(np.mean(its))}
    print(json.dumps(line))


def workload_serving(args):
    """Poisson arrivals (2000 req/s) of 9-point convection-diffusion (ILU(0)-
    BiCGSTAB, fp64) and 3D Poisson (SSOR-PCG, fp32 + refinement) requests
    through the solve server; solves/s and p50/p99 latency."""
    torch, nd, W = _setup()
    import numpy as np
    count = args.serving_requests
    t_arr, specs = W.serving_trace(count, 2000.0, 1005)
    reqs = []
    for sp in specs:
        r = W.build_request(sp)
        n = r["n"][0]
        if r["stencil"] == 9:
            k = max(1, -(-n // 128))
            r["sub"] = (k, k, 1)
            kw = dict(method=nd.BICGSTAB, precond=nd.PREC_ILU0, precision="fp64")
        else:
            k = max(1, -(-n // 32))
            r["sub"] = (k, k, k)
            kw = dict(method=nd.PCG, precond=nd.PREC_SSOR, precision="fp32")
        reqs.append((r, kw))
    S = nd.Server(slots=8)
    t0 = time.perf_counter()
    tickets = []
    for k in range(count):
        d = t0 + t_arr[k] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(S.submit(reqs[k][0], **reqs[k][1]))
    res = [S.wait(t, timeout=1800) for t in tickets]
    span = time.perf_counter() - t0
    st = S.stats()
    S.close()
    lat = np.array([r["latency_s"] for r, _ in res])
    # the 9-point sweep alone: ILU(0) applies of the largest request size
    n9 = 2048
    h9 = nd.NDiag(2, (n9, n9), 9, W.convdiff9(n9, 6.0, 1.1), (16, 16), "fp64")
    h9.ilu0_factor(nd.DECOMPOSED_FULL)  # the served factor
    r9 = torch.tensor(W.uniform_rhs(n9 * n9, 5), device="cuda")
    z9 = torch.empty_like(r9)
    for _ in range(2):
        h9.ilu0_apply(r9, z9)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        h9.ilu0_apply(r9, z9)
    e1.record()
    torch.cuda.synchronize()
    h9.close()
    ms9 = e0.elapsed_time(e1) / 5
    bytes9 = n9 * n9 * ((5 * 8 + 2 * 8) + (4 * 8 + 2 * 8))  # forward inv, 4 entries, r, y; backward 4 entries, y, z
    peak, kind = measured_peaks()
    gbs9 = bytes9 / (ms9 / 1e3) / 1e9
    print(json.dumps({"workload": f"serving-{count}-requests-poisson-arrivals-2000/s",
                      "metric": "solves/s; p50/p99 latency at rel-res 1e-8",
                      "solves_per_s": count / span, "p50_latency_s": float(np.percentile(lat, 50)),
                      "p99_latency_s": float(np.percentile(lat, 99)),
                      "ok": sum(r["status"] == "OK" for r, _ in res),
                      "relres_max": max(r["relres"] for r, _ in res), "max_running": st["max_running"],
                      "ninept_ilu_apply_2048": {"ms": ms9, "roofline": {
                          "bound": "hbm", "achieved": gbs9, "peak": peak, "unit": "GB/s", "frac": gbs9 / peak,
                          "peak_kind": kind, "kernel": "sweep9w_kernel (wavefront; ILU(0) forward and backward, fp64)"}}}))


def workload_mg2048(args):
    """The 2048^2 variable-coefficient workload (16 x 16 subdomains) solved by
    PCG with one multigrid V-cycle per iteration, the decomposed SSOR apply
    (omega 0.9) smoothing every level; beside it one BiCGSTAB + decomposed
    ILU(0) solve of the same system. V-cycle time with CUDA events around whole
    cycles."""
    import numpy as np
    torch, nd, W = _setup()
    p = W.varcoef2d_problem()
    n, om = p["n"][0], 0.9
    h = nd.NDiag(2, p["n"], 5, p["diags"], p["sub"], "fp64")
    b = torch.tensor(p["b"], device="cuda")
    r = b.clone()
    z = torch.empty_like(r)
    for _ in range(max(3, args.warmup)):
        h.mg_apply(om, r, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        h.mg_apply(om, r, z)
    e1.record()
    torch.cuda.synchronize()
    vc_ms = e0.elapsed_time(e1) / 10
    levels = h.mg_levels()
    # algorithmic bytes of one cycle, per cell of a level: two SSOR applies
    # (forward: pivot, 2 entries, r, tmp; backward: 2 entries, tmp, z) = 2 x 72,
    # two residuals (5 entries, b, x, r) = 2 x 64, restriction 10, prolongation
    # 18, the post-smoothing add 24; the coarsest level: 4 applies, 3 residuals,
    # 3 adds
    sizes, nx, ny = [], n, n
    for _ in range(levels):
        sizes.append(nx * ny)
        nx, ny = (nx + 1) // 2, (ny + 1) // 2
    vc_bytes = sum(c * 324 for c in sizes[:-1]) + sizes[-1] * (4 * 72 + 3 * 64 + 3 * 24)
    peak, kind = measured_peaks()
    gbs = vc_bytes / (vc_ms / 1e3) / 1e9
    walls = []
    for k in range(args.warmup + max(1, args.steps)):
        x = torch.zeros_like(b)
        info = _timed_solve(torch, h, nd.PCG, nd.PREC_MG, b, x, rtol=1e-8, maxit=2000, omega=om)
        if k >= args.warmup:
            walls.append(info["wall_s"])
    h.ilu0_factor()
    x = torch.zeros_like(b)
    ilu = _timed_solve(torch, h, nd.BICGSTAB, nd.PREC_ILU0, b, x, rtol=1e-8, maxit=20000)
    h.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        import oracle.mg as omg
        oracle.build()
        H = omg.Hierarchy(n, n, p["diags"], p["sub"], om)
        t0 = time.perf_counter()
        H.vcycle(p["b"])
        dt = time.perf_counter() - t0
        cpu = {"value": dt * 1e3, "unit": "ms per V-cycle", "cores": 1, "kind": "oracle",
               "sample": f"one V-cycle of the oracle (oracle/mg.py) on the same 2048^2 hierarchy ({dt:.1f} s)"}
    print(json.dumps({"workload": f"varcoef2d-{n}x{n}-5pt-fp64-mg-pcg-16x16", "metric": "solve seconds to rel-res 1e-8",
                      "mg_pcg": {"iters": info["iters"], "relres": info["relres"], "wall_s": float(np.median(walls)),
                                 "levels": levels, "omega": om, "vcycle_ms": vc_ms},
                      "vcycle_roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                          "frac": gbs / peak, "peak_kind": kind,
                                          "kernel": "one V-cycle (sweep2d SSOR applies, residuals, transfers)"},
                      "bicgstab_ilu0": {k: ilu[k] for k in ("iters", "relres", "wall_s")}, "cpu_baseline": cpu}))


def workload_eikonal2048(args):
    """Fast sweeping for |grad u| = f on 2048^2 cells (h = 1/2048, smoothed
    lognormal slowness, 4 point sources), 16 x 16 subdomains: whole solves to a
    round of four sweeps with no change (device vector; and from a host vector,
    copies included), and the time of one sweep with CUDA events around 20."""
    import numpy as np
    torch, nd, W = _setup()
    p = W.eikonal_problem()
    n = p["n"][0]
    e = nd.Eikonal(p["n"], p["h"], p["f"], p["sub"])
    a = torch.tensor(p["u0"], device="cuda")
    b = torch.empty_like(a)
    for t in range(4):
        e.sweep(t, a, b, wait=False)
        a, b = b, a
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for t in range(20):
        e.sweep(t, a, b, wait=False)
        a, b = b, a
    e1.record()
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1) / 20
    walls, host_walls = [], []
    for k in range(args.warmup + max(1, args.steps)):
        u = torch.tensor(p["u0"], device="cuda")
        torch.cuda.synchronize()
        info = e.solve(u)
        uh = p["u0"].copy()
        hinfo = e.solve(uh)
        if k >= args.warmup:
            walls.append(info["seconds"])
            host_walls.append(hinfo["seconds"])
    e.close()
    N = n * n
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        E = oracle.Eikonal(p["n"], p["h"], p["f"], p["sub"])
        u = p["u0"]
        t0 = time.perf_counter()
        for t in range(8):
            u, _ = E.sweep(t, u)
        dt = (time.perf_counter() - t0) / 8
        cpu = {"value": N / dt / 1e9, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"8 decomposed sweeps of the oracle on the same 2048^2 problem ({dt * 1e3:.0f} ms each)"}
    peak, kind = measured_peaks()
    gbs = 24.0 * N / (sweep_ms / 1e3) / 1e9  # u_old and f read, u_new written, 8 B each
    # the update is fp64 arithmetic: 14 operations a cell on its two-sided
    # branch (4 min, 4 mul, 4 add/sub, compare, sqrt), against the nominal
    # fp64 rate of 1.25 TFLOP/s = 625 G operations/s
    gops = 14.0 * N / (sweep_ms / 1e3) / 1e9
    print(json.dumps({"workload": f"eikonal2d-{n}x{n}-fast-sweeping-fp64-16x16", "metric":
                      "solve seconds (rounds of 4 sweeps until one changes nothing)",
                      "sweeps": info["sweeps"], "wall_s": float(np.median(walls)),
                      "e2e_host_wall_s": float(np.median(host_walls)), "sweep_ms": sweep_ms,
                      "gcell_updates_per_s": N / (sweep_ms / 1e3) / 1e9,
                      "roofline": {"bound": "alu", "achieved": gops, "peak": 625.0, "unit": "Gop/s (fp64)",
                                   "frac": gops / 625.0, "peak_kind": "nominal fp64 rate",
                                   "kernel": "eik_sweep_kernel"},
                      "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": kind},
                      "cpu_baseline": cpu}))


def workload_mg3d(args):
    """The 256^3 Poisson workload (8 x 8 x 8 subdomains, fp64) solved by PCG
    with the 3D multigrid V-cycle (decomposed SSOR smoother, omega 0.9), beside
    SSOR-PCG on the same handle. V-cycle time with CUDA events around whole
    cycles."""
    import numpy as np
    torch, nd, W = _setup()
    n = args.n3d
    p = W.poisson3d_problem(n, max(1, n // 32))
    om = 0.9
    h = nd.NDiag(3, p["n"], 7, p["diags"], p["sub"], "fp64")
    b = torch.tensor(p["b"], device="cuda")
    z = torch.empty_like(b)
    for _ in range(3):
        h.mg_apply(om, b, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        h.mg_apply(om, b, z)
    e1.record()
    torch.cuda.synchronize()
    vc_ms = e0.elapsed_time(e1) / 5
    walls = []
    for k in range(args.warmup + max(1, args.steps)):
        x = torch.zeros_like(b)
        info = _timed_solve(torch, h, nd.PCG, nd.PREC_MG, b, x, rtol=1e-8, maxit=500, omega=om)
        if k >= args.warmup:
            walls.append(info["wall_s"])
    x = torch.zeros_like(b)
    ssor = _timed_solve(torch, h, nd.PCG, nd.PREC_SSOR, b, x, rtol=1e-8, maxit=5000)
    levels = h.mg_levels()
    h.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        import oracle.mg as omg
        oracle.build()
        H = omg.Hierarchy3(p["n"], p["diags"], p["sub"], om)
        t0 = time.perf_counter()
        H.vcycle(p["b"])
        dt = time.perf_counter() - t0
        cpu = {"value": dt * 1e3, "unit": "ms per V-cycle", "cores": 1, "kind": "oracle",
               "sample": f"one V-cycle of the oracle (oracle/mg.py) on the same {n}^3 hierarchy ({dt:.1f} s)"}
    print(json.dumps({"workload": f"poisson3d-{n}^3-7pt-fp64-mg-pcg-{max(1, n // 32)}^3",
                      "metric": "solve seconds to rel-res 1e-8",
                      "mg_pcg": {"iters": info["iters"], "relres": info["relres"], "wall_s": float(np.median(walls)),
                                 "levels": levels, "omega": om, "vcycle_ms": vc_ms},
                      "ssor_pcg": {k: ssor[k] for k in ("iters", "relres", "wall_s")}, "cpu_baseline": cpu}))



def workload_convdiff9(args):
    """The largest served 9-point request: 2048^2 nonsymmetric convection-
    diffusion (Peclet 6, angle 1.1), 16 x 16 subdomains, fp64 BiCGSTAB with the
    decomposed full ILU(0) (and with D-ILU) to rel-res 1e-8; the ILU(0) apply
    timed with CUDA events for the wavefront and the level kernels.
    --kernel-only K: factor, then K applies (for kernel profiling)."""
    torch, nd, W = _setup()
    n = 2048
    d = W.convdiff9(n, 6.0, 1.1)
    b = torch.tensor(W.uniform_rhs(n * n, 5), device="cuda")
    peak, kind = measured_peaks()
    if args.kernel_only:
        h = nd.NDiag(2, (n, n), 9, d, (16, 16), "fp64")
        h.ilu0_factor(nd.DECOMPOSED_FULL)
        z = torch.empty_like(b)
        for _ in range(args.kernel_only):
            h.ilu0_apply(b, z)
        torch.cuda.synchronize()
        h.close()
        print(json.dumps({"workload": "convdiff9-2048^2-kernel-only", "applies": args.kernel_only}))
        return
    # bytes of one apply per cell: forward inv, 4 entries, r, y; backward 4 entries, y, z
    bpc = (5 * 8 + 2 * 8) + (4 * 8 + 2 * 8)
    out = {"workload": "convdiff9-2048^2-pe6-16x16-fp64-bicgstab-ilu0", "metric": "solve seconds; apply GB/s"}
    for name, mode, wave in (("full_ilu0", nd.DECOMPOSED_FULL, True), ("dilu", nd.DECOMPOSED, True),
                             ("full_ilu0_level_kernel", nd.DECOMPOSED_FULL, False)):
        h = nd.NDiag(2, (n, n), 9, d, (16, 16), "fp64")
        h.set_wavefront(wave)
        h.ilu0_factor(mode)
        z = torch.empty_like(b)
        for _ in range(3):
            h.ilu0_apply(b, z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            h.ilu0_apply(b, z)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        gbs = bpc * n * n / (ms / 1e3) / 1e9
        rec = {"apply_ms": ms, "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                            "frac": gbs / peak, "bytes_per_cell": bpc, "peak_kind": kind}}
        if name != "full_ilu0_level_kernel" or not args.no_natural:
            x = torch.zeros_like(b)
            info = _timed_solve(torch, h, nd.BICGSTAB, nd.PREC_ILU0, b, x, rtol=1e-8, maxit=20000)
            rec.update(iters=info["iters"], relres=info["relres"], seconds=info["wall_s"])
        h.close()
        out[name] = rec
    print(json.dumps(out))

EXTRA = {"poisson64": workload_poisson64, "poisson3d": workload_poisson3d,
         "batch512": workload_batch512, "serving": workload_serving, "mg2048": workload_mg2048,
         "eikonal2048": workload_eikonal2048, "mg3d": workload_mg3d, "convdiff9": workload_convdiff9}


if __name__ == "__main__":
    main()
