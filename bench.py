#!/usr/bin/env python
"""Benchmark: milliseconds to a 1e-10 relative residual on the 1M-vertex
jittered torus (A = M + 1e-4 L, cotan Laplacian, lumped mass), plus HBM GB/s
per V-cycle, against the plain FP64 GPU V-cycle.

One step = the numeric hierarchy setup of Alg. 1 for the step's matrix values
(Galerkin products A_{l+1} = P_l^T A_l P_l, the explicit inverse of the coarsest operator) and
the solve from x = 0 to ||b - A x|| <= 1e-10 ||b|| (FP64 conjugate gradients
preconditioned by one FP32 V-cycle per iteration).  The plain FP64 V-cycle
iteration of Alg. 1 and FP32-cycle iterative refinement are timed on the same
hierarchy and reported beside it.  The hierarchy topology (P_l, colourings,
patterns, launch shapes) is set up once before timing.  Inputs are resident in HBM when the timed region
starts; L2 is flushed (256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmg|reference]

With --impl reference the CPU FP64 oracle is timed on the same workload (one
full setup + solve per step, on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to 1e-10 rel. residual and HBM GB/s per V-cycle vs plain FP64 GPU V-cycle"
WORKLOAD = "torus1m"
WORKLOAD_DESC = ("jittered torus 2048x512 (1,048,576 vertices, R=1, r=0.3, jitter 0.2 edge, seed 1), "
                 "cotan L, lumped M, (M + 1e-4 L) x = M b, b ~ N(0,1)")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest value over the ranks of the job (one replica per GPU; the
    slowest replica sets the job's time), or the value itself with one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def mark(self, timeout_s: float = 5.0):
        """Waits for the first sample, then marks the start of the timed region
        (the last sample before it still counts: it is the state the region
        starts in)."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)
        self.i0 = max(0, len(self.lines) - 1)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "i0", 0):]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(dims, Ps, s):
    """Algorithmic bytes of one V-cycle with nu = 2/2 (each value read or
    written once per pass, 4-byte indices): per level l < lambda,
    5 [z_l (s+4) + 4 n_l] + 15 n_l s + [3 n_l (4+s) + n_l s + n_{l+1} s + 4 n_{l+1}]
    + [3 n_l (4+s) + n_{l+1} s + 2 n_l s]; the coarsest level adds n^2 * 8 (FP64 inverse)."""
    total = 0.0
    for l in range(len(dims) - 1):
        n, z, _ = dims[l]
        nc = dims[l + 1][0]
        total += 5 * (z * (s + 4) + 4 * n) + 15 * n * s
        total += 3 * n * (4 + s) + n * s + nc * s + 4 * nc
        total += 3 * n * (4 + s) + nc * s + 2 * n * s
    nl = dims[-1][0]
    total += nl * nl * 8
    return total


def gs_launch_bytes(dims, s):
    """Average algorithmic bytes of one finest-level Gauss-Seidel colour
    launch: per sweep z_off (s + 4) [values + indices] + 3 n s [b, 1/a_ii, x
    write] + (C - 1) n s [x of the other colours, read once per launch];
    divided by the C colour launches of a sweep."""
    n, z, C = dims[0]
    sweep = (z - n) * (s + 4) + 3 * n * s + (C - 1) * n * s
    return sweep / C


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of `kernel` on `workload` from the committed ncu capture summary, or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        return d.get(workload, {}).get(kernel)
    except Exception:
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import gmg_inputs as gi
    import oracle

    oracle.compile_oracle()
    s = gi.workload(WORKLOAD)
    times, iters = [], 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = oracle.Oracle(s.A, s.Ps)
        x, iters, hist, ok = o.solve(s.b, tol=1e-10, max_iter=200, pcg=True)
        dt = (time.perf_counter() - t0) * 1e3
        del o
        if k >= args.warmup:
            times.append(dt)
    ms = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "solver": "CPU FP64 oracle: Galerkin setup + Cholesky + V-cycle-preconditioned CG",
                   "iterations": iters},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full oracle runs (setup + {iters} PCG iterations to 1e-10)"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(s):
    import oracle

    oracle.compile_oracle()
    t0 = time.perf_counter()
    o = oracle.Oracle(s.A, s.Ps)
    x, iters, hist, ok = o.solve(s.b, tol=1e-10, max_iter=200, pcg=True)
    ms = (time.perf_counter() - t0) * 1e3
    return {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"one full oracle run on the same system: Galerkin setup + Cholesky + {iters} FP64 "
                      f"V-cycle-preconditioned CG iterations to 1e-10, single thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmg", choices=["gmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="set up, autotune, run `warmup` untimed steps and one step, print a short note and exit "
                         "(the launch sequence a kernel profiler lists; no timing is reported)")
    ap.add_argument("--lanes", default=None,
                    help="comma-separated warps-per-row split of every smoothed level (instead of the autotuner)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import gmg_inputs as gi
    import paper_2307_04886_gb300 as g

    g.build_library()
    s = gi.workload(WORKLOAD)
    A = s.A
    n = A.shape[0]

    t0 = time.perf_counter()
    solver = g.Solver(A, s.Ps, precision=g.GMG_FP32_PCG)
    if args.lanes:
        lanes = [int(v) for v in args.lanes.split(",")]
        solver.set_lanes(lanes)
    else:
        lanes = solver.autotune()
    torch.cuda.synchronize()
    symbolic_ms = (time.perf_counter() - t0) * 1e3
    dims = solver.dims

    vals = torch.tensor(A.data, device=dev)
    b = torch.tensor(s.b, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(sv):
        sv.set_values(vals)
        x.zero_()
        return sv.solve(b, x, tol=1e-10)

    def timed(sv, steps, warmup, prof=False, clk=None):
        for _ in range(warmup):
            step(sv)
        torch.cuda.synchronize()
        if clk is not None:
            clk.mark()
        if ws > 1:
            torch.distributed.barrier()
        if prof:
            sv.profile(True)
            sv.profile_read()
        l0 = g.kernel_launches()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            _, iters, rr, _, _ = step(sv)
            evs[k][1].record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - w0) * 1e3
        launches = g.kernel_launches() - l0
        ms = [a.elapsed_time(bb) for a, bb in evs]
        pr = sv.profile_read() if prof else None
        if prof:
            sv.profile(False)
        return sum(ms) / steps, iters, rr, launches, pr, wall

    if args.profile_step:
        for _ in range(args.warmup + 1):
            step(solver)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "workload": WORKLOAD, "warps_per_row": lanes,
                          "kernel_launches_total": g.kernel_launches()}), flush=True)
        solver.close()
        return 0

    clk = ClockSampler(dev.index)
    clk.start()
    ms, iters, rr, launches, _, wall = timed(solver, args.steps, args.warmup, prof=False, clk=clk)
    clocks = clk.stop()
    # per-kernel timing (CUDA events around the finest smoothing blocks and each
    # V-cycle) runs the host-driven loop: event nodes cannot sit in the device loop
    _, _, _, _, pr, _ = timed(solver, 5, 1, prof=True)
    ms = max_over_ranks(ms, dev)

    # breakdown (not part of the headline): numeric setup alone
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        solver.set_values(vals)
    e1.record()
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1) / 5

    # the plain FP64 V-cycle and FP32-cycle iterative refinement on the same hierarchy
    others = {}
    for name, prec in (("fp64_plain", g.GMG_FP64), ("fp32_refine", g.GMG_FP32_REFINE)):
        sv = g.Solver(A, s.Ps, precision=prec)
        sv.set_lanes(lanes)
        o_ms, o_it, _, _, _, _ = timed(sv, max(2, args.steps // 2), 3)
        _, _, _, _, o_pr, _ = timed(sv, 3, 1, prof=True)
        others[name] = (o_ms, o_it, o_pr)
        sv.close()

    # end to end through the C ABI with host buffers (pinned), copies inside
    vals_h = torch.tensor(A.data).pin_memory().numpy()
    b_h = torch.tensor(s.b).pin_memory().numpy()
    for _ in range(2):
        solver.set_values(vals_h)
        solver.solve(b_h, None, tol=1e-10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        solver.set_values(vals_h)
        xh, _, _, _, _ = solver.solve(b_h, None, tol=1e-10)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps

    # roofline of the dominant kernel: finest-level FP32 Gauss-Seidel colour launch
    peak, peak_kind = load_peaks()
    smooth_ms, gs_launches, cyc_ms, cycles = pr
    gs_avg_ms = smooth_ms / max(gs_launches, 1)
    gs_bytes = gs_launch_bytes(dims, 4)
    achieved = gs_bytes / (gs_avg_ms * 1e-3) / 1e9
    vc_bytes32 = algorithmic_bytes(dims, s.Ps, 4)
    vc_gbs = vc_bytes32 / (cyc_ms / max(cycles, 1) * 1e-3) / 1e9
    vc_bytes64 = algorithmic_bytes(dims, s.Ps, 8)
    f_ms, f_it, f_pr = others["fp64_plain"]
    r_ms, r_it, r_pr = others["fp32_refine"]
    vc64_us = 1e3 * f_pr[2] / max(f_pr[3], 1)
    traffic = ncu_traffic(f"k_gs<float, {lanes[0]}>", WORKLOAD)

    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_DESC, "levels": [d[0] for d in dims], "nnz": [d[1] for d in dims],
            "colours": [d[2] for d in dims], "warps_per_row": lanes,
            "precision": "FP64 conjugate gradients preconditioned by one FP32 V-cycle (nu=2/2, multicolour GS) "
                         "per iteration; FP64 residual, dots and explicit coarsest inverse; the iterations run in a device-side "
                         "graph loop (conditional WHILE node)",
            "iterations": iters, "final_rel_res": rr,
            "step": "numeric Galerkin setup + coarsest inverse + solve from x=0 to 1e-10",
            "l2": "flushed before every timed step (256 MB write)",
            "numeric_setup_ms": setup_ms, "solve_ms": ms - setup_ms, "symbolic_setup_ms": symbolic_ms,
            "fp64_plain_ms": f_ms, "fp64_plain_iterations": f_it,
            "fp32_refine_ms": r_ms, "fp32_refine_iterations": r_it,
            "speedup_vs_fp64_plain": f_ms / ms,
            "vcycle_us_fp32": 1e3 * cyc_ms / max(cycles, 1), "vcycle_gbs_fp32": vc_gbs,
            "vcycle_bytes_fp32": vc_bytes32, "vcycle_us_fp64": vc64_us,
            "vcycle_gbs_fp64": vc_bytes64 / (vc64_us * 1e-6) / 1e9, "vcycle_bytes_fp64": vc_bytes64,
            "wall_ms_timed_region": wall,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
        },
        "roofline": {"bound": "hbm", "kernel": f"k_gs<float, {lanes[0]}> (finest level, one colour)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "bytes_per_launch": gs_bytes, "avg_launch_us": gs_avg_ms * 1e3},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(A.data.nbytes + s.b.nbytes),
                "d2h_bytes_per_step": int(8 * n)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s)
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
