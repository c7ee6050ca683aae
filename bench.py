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
full setup + solve per step, on all host cores).

Beside the headline the JSON line carries, under config.workloads, the other
synthetic workloads measured on the same GPU (--configs none skips them):
icosphere5 (plain FP64 V-cycle iteration), heat512k (forward + adjoint solve of
the differentiable heat diffusion), book5 (smoothing on a non-manifold mesh),
spheres64 (64 meshes x 8 right-hand sides in one many-mesh solve against 512
plain FP64 single solves) and cloud4m (the 4M-point kNN cloud, with
Gauss-Seidel GB/s per level).
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


def gs_level_launch_bytes(dims, l, s):
    """Average algorithmic bytes of one Gauss-Seidel colour launch on level l
    (the formula of gs_launch_bytes on that level's rows, entries, colours)."""
    n, z, C = dims[l]
    return ((z - n) * (s + 4) + 3 * n * s + (C - 1) * n * s) / C


def gs_kernel_name(split, t="float"):
    return f"k_gs<{t}, {split}>"


def level_breakdown(dims, lanes, levels, cycles, s=4, paths=None):
    """Per smoothed level of the timed cycles: Gauss-Seidel launches, average
    launch time and algorithmic GB/s, the transfer (residual, restriction,
    prolongation) time, and the cluster tail (levels it covers, time).  A
    cluster level (paths[l] == 1) runs its sweeps and transfers in two cluster
    launches: its time per Gauss-Seidel phase includes the transfers."""
    out, tail = [], None
    cyc = max(cycles, 1)
    for l, (gs_ms, gs_n, tr_ms, whole_ms) in enumerate(levels):
        if l >= len(dims) - 1:
            break
        if gs_n > 0:
            us = 1e3 * gs_ms / gs_n
            b = gs_level_launch_bytes(dims, l, s)
            kern = "k_level_cluster" if paths and paths[l] == 1 else gs_kernel_name(lanes[l])
            out.append({"level": l, "rows": dims[l][0], "colours": dims[l][2], "kernel": kern,
                        "gs_launches_per_cycle": gs_n / cyc, "gs_us_per_launch": us,
                        "gs_bytes_per_launch": b, "gs_gbs": b / (us * 1e-6) / 1e9,
                        "gs_us_per_cycle": 1e3 * gs_ms / cyc, "transfer_us_per_cycle": 1e3 * tr_ms / cyc})
        elif whole_ms > 0 and tail is None:
            tail = {"kernel": "k_tail_cycle", "levels": list(range(l, len(dims))), "us_per_cycle": 1e3 * whole_ms / cyc}
    return out, tail


def dominant_gs(per_level):
    """The Gauss-Seidel kernel instantiation with the largest time per cycle,
    summed over the levels that run it: (name, us per launch, bytes per launch,
    us per cycle)."""
    groups = {}
    for r in per_level:
        g = groups.setdefault(r["kernel"], [0.0, 0.0, 0.0, []])
        g[0] += r["gs_us_per_cycle"]
        g[1] += r["gs_launches_per_cycle"]
        g[2] += r["gs_bytes_per_launch"] * r["gs_launches_per_cycle"]
        g[3].append(r["level"])
    name, (us_cyc, n_cyc, bytes_cyc, lv) = max(groups.items(), key=lambda kv: kv[1][0])
    return name, us_cyc / n_cyc, bytes_cyc / n_cyc, us_cyc, lv


def ncu_traffic(workload, per_level, levels, kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    the Gauss-Seidel launches on `levels` of `workload`, from the committed ncu
    capture summary (bytes per launch for each level), weighted by each level's
    launches per V-cycle as the algorithmic bytes are; None if a level is missing."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            j = json.load(f)[workload]
        if kernel == "k_level_cluster":  # the two launches of a V-cycle, per Gauss-Seidel phase like the bytes
            r = next(r for r in per_level if r["level"] in levels)
            return float(j["cluster_level_bytes_per_cycle"]) / r["gs_launches_per_cycle"]
        if not kernel.startswith("k_gs<"):
            return None
        d = j["gs_bytes_per_launch_by_level"]
        num = den = 0.0
        for r in per_level:
            if r["level"] in levels:
                num += r["gs_launches_per_cycle"] * float(d[str(r["level"])])
                den += r["gs_launches_per_cycle"]
        return num / den if den else None
    except Exception:
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def oracle_step(s, lib_path=None):
    """One oracle step on system s: the full setup of Alg. 1 (Galerkin levels,
    colourings, Cholesky) and the V-cycle-preconditioned CG solve to 1e-10.
    Returns (setup ms, solve ms, iterations)."""
    import oracle

    t0 = time.perf_counter()
    o = oracle.Oracle(s.A, s.Ps, lib_path=lib_path)
    t1 = time.perf_counter()
    x, iters, hist, ok = o.solve(s.b, tol=1e-10, max_iter=200, pcg=True)
    t2 = time.perf_counter()
    del o
    return (t1 - t0) * 1e3, (t2 - t1) * 1e3, iters


def threaded_oracle():
    """(library path, cores) of the all-cores oracle build, or (None, 1)."""
    import oracle

    path = oracle.compile_oracle_threaded()
    return (path, oracle.host_cores()) if path else (None, 1)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import gmg_inputs as gi
    import oracle

    oracle.compile_oracle()
    path, cores = threaded_oracle()
    s = gi.workload(WORKLOAD)
    times, setups, solves, iters = [], [], [], 0
    for k in range(args.warmup + args.steps):
        su, so, iters = oracle_step(s, path)
        if k >= args.warmup:
            times.append(su + so)
            setups.append(su)
            solves.append(so)
    ms = sum(times) / len(times)
    # one V-cycle of the oracle alone (FP64, from x = 0), as the paper times its cycles
    o = oracle.Oracle(s.A, s.Ps, lib_path=path)
    x0 = np.zeros(s.n)
    o.vcycle(x0, s.b)
    t0 = time.perf_counter()
    for _ in range(3):
        o.vcycle(x0, s.b)
    vcycle_ms = (time.perf_counter() - t0) * 1e3 / 3
    del o
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC,
                   "solver": "CPU FP64 oracle: Galerkin setup + colouring + Cholesky + V-cycle-preconditioned CG",
                   "iterations": iters, "setup_ms": sum(setups) / len(setups),
                   "solve_ms": sum(solves) / len(solves), "vcycle_ms": vcycle_ms},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full oracle runs (setup + {iters} PCG iterations to 1e-10) on "
                                   f"{cores} host threads (OpenMP over independent rows)"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(s):
    """The oracle on the same system: all host cores (the threaded build) and
    one thread (the paper's setting), one full step each."""
    import oracle

    oracle.compile_oracle()
    path, cores = threaded_oracle()
    su1, so1, it1 = oracle_step(s)
    out = {"unit": "ms", "kind": "oracle",
           "single_thread": {"value": su1 + so1, "setup_ms": su1, "solve_ms": so1, "cores": 1}}
    if path:
        su, so, it = oracle_step(s, path)
        out.update(value=su + so, cores=cores, setup_ms=su, solve_ms=so,
                   sample=f"one full oracle step on the same system (Galerkin setup + colouring + Cholesky + {it} "
                          f"FP64 V-cycle-preconditioned CG iterations to 1e-10) on {cores} host threads; "
                          f"single_thread: the same step on one thread")
    else:
        out.update(value=su1 + so1, cores=1,
                   sample=f"one full oracle step on one thread ({it1} PCG iterations); no OpenMP runtime")
    return out


def _ev_ms(fn, reps):
    """Average ms of fn() over reps runs, timed with CUDA events on the current stream."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def other_workloads(g, names, steps):
    """Timings of the other synthetic workloads (each inputs-resident, events
    on the solve stream); a workload that cannot be set up is reported with
    its error."""
    import numpy as np
    import torch

    import gmg_inputs as gi

    dev = torch.device("cuda", torch.cuda.current_device())
    res = {}
    for name in names:
        t0 = time.perf_counter()
        try:
            if name == "icosphere5":
                s = gi.workload(name)
                b = torch.tensor(s.b, device=dev)
                x = torch.zeros_like(b)
                r = {"rows": s.n}
                for tag, prec in (("fp64_plain", g.GMG_FP64), ("fp32_pcg", g.GMG_FP32_PCG)):
                    sv = g.Solver(s.A, s.Ps, precision=prec)
                    sv.autotune()
                    out = {}

                    def run():
                        x.zero_()
                        out["r"] = sv.solve(b, x, tol=1e-10)

                    _ev_ms(run, 3)
                    r[f"{tag}_ms"] = _ev_ms(run, steps)
                    r[f"{tag}_iterations"] = out["r"][1]
                    sv.close()
                res[name] = r
            elif name == "heat512k":
                s = gi.workload(name)
                sv = g.Solver(None, s.Ps, precision=g.GMG_FP32_PCG, ml=(s.Mdiag, s.L, s.t))
                sv.autotune()
                u0 = torch.tensor(s.extra["u0"], device=dev)
                xt = torch.tensor(s.extra["x_target"], device=dev)
                x, lam = torch.zeros_like(u0), torch.zeros_like(u0)
                it = {}

                def fwd_adj():
                    sv.set_t(s.t)
                    bb = sv.mass(u0)
                    x.zero_()
                    it["f"] = sv.solve(bb, x, tol=1e-10)[1]
                    lam.zero_()
                    it["a"] = sv.solve(2.0 * (x - xt), lam, tol=1e-10)[1]
                    sv.grad(lam, x)

                _ev_ms(fwd_adj, 2)
                res[name] = {"rows": s.n, "forward_adjoint_ms": _ev_ms(fwd_adj, steps),
                             "step": "set_t (numeric refresh) + M u0 + forward solve + adjoint solve + gradient kernel",
                             "forward_iterations": it["f"], "adjoint_iterations": it["a"], "tol": 1e-10}
                sv.close()
            elif name == "spheres64":
                systems = gi.cached_batch("spheres64", gi.spheres_batch)
                many = g.SolverMany([(q.A, q.Ps) for q in systems])
                many.autotune(int(systems[0].b.shape[1]))  # multi-right-hand-side row splits per mesh and level
                Bs = [torch.tensor(q.b, device=dev) for q in systems]
                Xs = [torch.zeros_like(B) for B in Bs]
                out = {}

                def run_many():
                    for X in Xs:
                        X.zero_()
                    out["m"] = many.solve(Bs, Xs, tol=1e-10)

                _ev_ms(run_many, 2)
                many_ms = _ev_ms(run_many, steps)
                its = out["m"][1]
                many.close()
                singles = [g.Solver(q.A, q.Ps, precision=g.GMG_FP64) for q in systems]
                cols = [[B[:, c].contiguous() for c in range(B.shape[1])] for B in Bs]
                xs = [torch.zeros_like(cs[0]) for cs in cols]

                def run_single():
                    for sv, cs, xx in zip(singles, cols, xs):
                        for bcol in cs:
                            xx.zero_()
                            sv.solve(bcol, xx, tol=1e-10)

                run_single()
                single_ms = _ev_ms(run_single, max(1, steps // 4))
                for sv in singles:
                    sv.close()
                res[name] = {"meshes": len(systems), "rows_total": int(sum(q.n for q in systems)),
                             "rhs_per_mesh": int(systems[0].b.shape[1]), "many_ms": many_ms,
                             "many_iterations_max": int(max(its)), "many_iterations_min": int(min(its)),
                             "plain_fp64_single_solves_ms": single_ms,
                             "speedup_vs_plain_fp64": single_ms / many_ms,
                             "plain": "every column solved alone by the plain FP64 V-cycle iteration (gmg_solve)",
                             "shapes": "multi-right-hand-side row splits autotuned per mesh and level"}
            elif name == "book5":
                s = gi.workload(name)
                b = torch.tensor(s.b, device=dev)
                x = torch.zeros_like(b)
                r = {"rows": s.n, "mesh": "non-manifold: 5 bent sheets sharing a spine (Sec. 5.4 stand-in)"}
                for tag, prec in (("fp64_plain", g.GMG_FP64), ("fp32_pcg", g.GMG_FP32_PCG)):
                    sv = g.Solver(s.A, s.Ps, precision=prec)
                    sv.autotune()
                    out = {}

                    def run():
                        x.zero_()
                        out["r"] = sv.solve(b, x, tol=1e-10)

                    _ev_ms(run, 3)
                    r[f"{tag}_ms"] = _ev_ms(run, steps)
                    r[f"{tag}_iterations"] = out["r"][1]
                    sv.close()
                res[name] = r
            elif name == "cloud4m":
                s = gi.workload(name)
                sv = g.Solver(s.A, s.Ps, precision=g.GMG_FP32_PCG)
                lanes = sv.autotune()
                b = torch.tensor(s.b, device=dev)
                x = torch.zeros_like(b)
                out = {}

                def run():
                    x.zero_()
                    out["r"] = sv.solve(b, x, tol=1e-10)

                _ev_ms(run, 2)
                ms = _ev_ms(run, steps)
                sv.profile(True)
                sv.profile_read()
                sv.profile_levels()
                for _ in range(2):
                    run()
                pr = sv.profile_read()
                lv = sv.profile_levels()
                sv.profile(False)
                per_level, tail = level_breakdown(sv.dims, lanes, lv, int(pr[3]), paths=sv.paths)
                res[name] = {"rows": s.n, "levels": [d[0] for d in sv.dims], "nnz": [d[1] for d in sv.dims],
                             "colours": [d[2] for d in sv.dims], "fp32_pcg_ms": ms, "iterations": out["r"][1],
                             "vcycle_us_fp32": 1e3 * pr[2] / max(pr[3], 1),
                             "vcycle_gbs_fp32": algorithmic_bytes(sv.dims, s.Ps, 4) / (pr[2] / max(pr[3], 1) * 1e-3) / 1e9,
                             "per_level": per_level, "tail": tail}
                sv.close()
        except Exception as e:  # reported, not fatal: the headline stands on its own
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        res.setdefault(name, {})["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
    return res


def profile_config(args):
    """One workload's solves for a kernel profiler: the launch sequence of the
    timed solve, with a fixed warps-per-row split instead of the autotuner."""
    import torch

    import gmg_inputs as gi
    import paper_2307_04886_gb300 as g

    g.build_library()
    torch.cuda.set_device(0)
    s = gi.workload(args.profile_config)
    sv = g.Solver(s.A, s.Ps, precision=g.GMG_FP32_PCG)
    if args.lanes:
        ln = [int(v) for v in args.lanes.split(",")]
        sv.set_lanes((ln + [ln[-1]] * len(sv.dims))[:max(1, len(sv.dims) - 1)])
    b = torch.tensor(s.b, device="cuda")
    x = torch.zeros_like(b)
    for _ in range(args.warmup + 1):
        x.zero_()
        r = sv.solve(b, x, tol=1e-10)
    torch.cuda.synchronize()
    print(json.dumps({"profile_config": args.profile_config, "levels": [d[0] for d in sv.dims],
                      "iterations": r[1], "level_paths": sv.paths}), flush=True)
    sv.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmg", choices=["gmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs", default="icosphere5,heat512k,book5,spheres64,cloud4m",
                    help="comma-separated other workloads to time after the headline, or 'none'; a trailing '?' "
                         "times that workload only when its inputs are already cached (cloud4m's take one to two "
                         "minutes to generate on the host, once)")
    ap.add_argument("--profile-step", action="store_true",
                    help="set up, autotune, run `warmup` untimed steps and one step, print a short note and exit "
                         "(the launch sequence a kernel profiler lists; no timing is reported)")
    ap.add_argument("--profile-config", default=None,
                    help="set up the named other workload (e.g. cloud4m) with the --lanes split, run `warmup` + 1 "
                         "solves to 1e-10, print a short note and exit (for kernel profilers; no timing)")
    ap.add_argument("--lanes", default=None,
                    help="comma-separated warps-per-row split of every smoothed level (instead of the autotuner)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_config:
        return profile_config(args)

    ws, rank, local = dist_env()
    # inputs of the other workloads that take long to generate, prepared by a
    # separate process while the headline runs
    names = [] if args.configs == "none" else [c for c in args.configs.split(",") if c]
    prep = None
    if rank == 0 and "spheres64" in names:
        prep = subprocess.Popen([sys.executable, "-c", "import gmg_inputs as gi; gi.cached_batch('spheres64', gi.spheres_batch)"],
                                cwd=ROOT, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)

    import numpy as np
    import torch

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

    # the first set-up in a process also loads the library's kernels and
    # creates the CUDA context; the second is what each new mesh pays
    t0 = time.perf_counter()
    solver = g.Solver(A, s.Ps, precision=g.GMG_FP32_PCG)
    torch.cuda.synchronize()
    first_setup_ms = (time.perf_counter() - t0) * 1e3
    solver.close()
    t0 = time.perf_counter()
    solver = g.Solver(A, s.Ps, precision=g.GMG_FP32_PCG)
    torch.cuda.synchronize()
    symbolic_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    if args.lanes:
        lanes = [int(v) for v in args.lanes.split(",")]
        solver.set_lanes(lanes)
    else:
        lanes = solver.autotune()
    torch.cuda.synchronize()
    autotune_ms = (time.perf_counter() - t0) * 1e3
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
            sv.profile_levels()
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
        lv = sv.profile_levels() if prof else None
        if prof:
            sv.profile(False)
        return sum(ms) / steps, iters, rr, launches, (pr, lv), wall

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
    # per-kernel timing (CUDA events around every level's smoothing blocks and
    # each V-cycle) runs the host-driven loop: event nodes cannot sit in the device loop
    _, _, _, _, (pr, lv), _ = timed(solver, 5, 1, prof=True)
    ms = max_over_ranks(ms, dev)

    # breakdown (not part of the headline): numeric setup alone
    torch.cuda.synchronize()
    setup_ms = []
    for _ in range(5):  # each refresh timed alone: the previous one's inverse has finished
        torch.cuda.synchronize()
        setup_ms.append(_ev_ms(lambda: solver.set_values(vals), 1))
    setup_ms = sorted(setup_ms)[len(setup_ms) // 2]
    # the same refresh until its coarsest inverse (second stream) is done: host clock to a device-wide sync
    setup_full_ms = []
    for _ in range(5):
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        solver.set_values(vals)
        torch.cuda.synchronize()
        setup_full_ms.append((time.perf_counter() - w0) * 1e3)
    setup_full_ms = sorted(setup_full_ms)[len(setup_full_ms) // 2]

    # the plain FP64 V-cycle, FP32-cycle iterative refinement and CG with the
    # FP64 cycle, on the same hierarchy
    others = {}
    for name, prec in (("fp64_plain", g.GMG_FP64), ("fp32_refine", g.GMG_FP32_REFINE), ("fp64_pcg", g.GMG_FP64_PCG)):
        sv = g.Solver(A, s.Ps, precision=prec)
        sv.set_lanes(lanes)
        o_ms, o_it, _, _, _, _ = timed(sv, max(2, args.steps // 2), 3)
        _, _, _, _, (o_pr, o_lv), _ = timed(sv, 3, 1, prof=True)
        others[name] = (o_ms, o_it, o_pr, o_lv)
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

    # roofline: the Gauss-Seidel kernel instantiation with the largest share of
    # the V-cycle (per-level CUDA events), and the whole V-cycle in each precision
    peak, peak_kind = load_peaks()
    smooth_ms, gs_launches, cyc_ms, cycles = pr
    cycles = int(cycles)
    per_level, tail = level_breakdown(dims, lanes, lv, cycles, paths=solver.paths)
    kname, k_us, k_bytes, k_us_cyc, k_levels = dominant_gs(per_level)
    achieved = k_bytes / (k_us * 1e-6) / 1e9
    vc_us32 = 1e3 * cyc_ms / max(cycles, 1)
    vc_bytes32 = algorithmic_bytes(dims, s.Ps, 4)
    vc_gbs32 = vc_bytes32 / (vc_us32 * 1e-6) / 1e9
    vc_bytes64 = algorithmic_bytes(dims, s.Ps, 8)
    f_ms, f_it, f_pr, f_lv = others["fp64_plain"]
    r_ms, r_it, r_pr, r_lv = others["fp32_refine"]
    p_ms, p_it, p_pr, p_lv = others["fp64_pcg"]
    vc_us64 = 1e3 * f_pr[2] / max(f_pr[3], 1)
    vc_gbs64 = vc_bytes64 / (vc_us64 * 1e-6) / 1e9
    per_level64, _ = level_breakdown(dims, lanes, f_lv, int(f_pr[3]), s=8)
    for r in per_level64:
        r["kernel"] = r["kernel"].replace("float", "double")
    traffic = ncu_traffic(WORKLOAD, per_level, k_levels, kname)

    # Sec. 4 hierarchy construction of the same mesh on the GPU, against the host builder
    build_info = None
    if rank == 0:
        try:
            from gmg_inputs import meshes, operators
            from gmg_inputs.hierarchy import build_hierarchy as host_build

            V, F, _ = meshes.jittered_torus(2048, 512, 1)
            rp, ci = operators.edges_to_adjacency(V.shape[0], meshes.mesh_edges(F))
            g.build_hierarchy(V, rp, ci)  # warm-up (module load, first allocations)
            w0 = time.perf_counter()
            lv, gpu_ms = g.build_hierarchy(V, rp, ci)
            wall_ms = (time.perf_counter() - w0) * 1e3
            w0 = time.perf_counter()
            hPs = host_build(V, rp, ci)
            host_ms = (time.perf_counter() - w0) * 1e3
            same = len(hPs) == len(lv) and all(
                np.array_equal(a.idx, b.idx) and np.array_equal(a.w, b.w) for a, b in zip(hPs, lv))
            build_info = {"gpu_ms": gpu_ms, "gpu_call_wall_ms": wall_ms, "host_builder_ms": host_ms,
                          "speedup": host_ms / wall_ms, "levels": [1048576] + [q.n_coarse for q in lv],
                          "prolongations_identical_to_host_builder": bool(same),
                          "what": "gmg_build_hierarchy (Sec. 4 sampling, Voronoi cells, coarse graph, triangles, "
                                  "barycentric prolongation) on the torus1m mesh, phi = 1/8, stop at 1000"}
        except Exception as e:
            build_info = {"error": f"{type(e).__name__}: {e}"}

    extra = {}
    if prep is not None:
        prep.wait()
    if names and rank == 0:
        chosen = []
        for nm in names:
            if nm.endswith("?"):
                nm = nm[:-1]
                if not gi.is_cached(nm):
                    extra[nm] = {"skipped": "inputs not cached on this machine (generating them takes minutes); "
                                            f"python bench.py --configs {nm} generates and times them"}
                    continue
            chosen.append(nm)
        extra.update(other_workloads(g, chosen, max(3, args.steps // 3)))

    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_DESC, "levels": [d[0] for d in dims], "nnz": [d[1] for d in dims],
            "colours": [d[2] for d in dims], "warps_per_row": lanes,
            "level_paths": solver.paths,
            "level_paths_legend": "FP32 cycle per level: 0 one launch per colour, 1 cluster level (two cluster "
                                  "launches), 2 cluster tail, 3 coarsest direct solve",
            "precision": "FP64 conjugate gradients preconditioned by one FP32 V-cycle (nu=2/2, multicolour GS) "
                         "per iteration; FP64 residual, dots and explicit coarsest inverse; the iterations run in a device-side "
                         "graph loop (conditional WHILE node)",
            "iterations": iters, "final_rel_res": rr,
            "step": "numeric Galerkin setup + coarsest inverse + solve from x=0 to 1e-10",
            "l2": "flushed before every timed step (256 MB write)",
            "numeric_setup_ms": setup_ms, "numeric_setup_with_inverse_wall_ms": setup_full_ms,
            "symbolic_setup_ms": symbolic_ms, "first_setup_in_process_ms": first_setup_ms,
            "symbolic_setup": "gmg_setup (validation, symbolic Galerkin product and plans, colourings, layouts, "
                              "cluster tables, first numeric set-up) on a process that has set up once before; "
                              "first_setup_in_process_ms includes CUDA context and kernel loading",
            "autotune_ms": autotune_ms,
            "numeric_setup": "gmg_set_values as its caller sees it: Galerkin values, solve layout and their checks; "
                             "the coarsest inverse runs on the handle's second stream, and the solve waits for it "
                             "right before its first coarse solve (inside the timed step); "
                             "numeric_setup_with_inverse_wall_ms: host clock from the call to a device-wide "
                             "synchronize after it (median of 5)",
            "fp64_plain_ms": f_ms, "fp64_plain_iterations": f_it,
            "fp32_refine_ms": r_ms, "fp32_refine_iterations": r_it,
            "fp64_pcg_ms": p_ms, "fp64_pcg_iterations": p_it,
            "speedup_vs_fp64_plain": f_ms / ms,
            "speedup_fp32_cycle_inside_cg": p_ms / ms,
            "speedup_cg_with_fp64_cycle_vs_fp64_plain": f_ms / p_ms,
            "vcycle_us_fp32": vc_us32, "vcycle_gbs_fp32": vc_gbs32,
            "vcycle_bytes_fp32": vc_bytes32, "vcycle_us_fp64": vc_us64,
            "vcycle_gbs_fp64": vc_gbs64, "vcycle_bytes_fp64": vc_bytes64,
            "per_level_fp32": per_level, "tail_fp32": tail, "per_level_fp64": per_level64,
            "wall_ms_timed_region": wall,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "workloads": extra,
            "hierarchy_build": build_info,
        },
        "roofline": {"bound": "hbm", "kernel": f"{kname} (levels {k_levels}, one colour per launch)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "bytes_per_launch": k_bytes,
                     "avg_launch_us": k_us, "us_per_vcycle": k_us_cyc, "share_of_vcycle": k_us_cyc / vc_us32,
                     "vcycle_fp32": {"achieved": vc_gbs32, "frac": vc_gbs32 / peak, "us": vc_us32},
                     "vcycle_fp64": {"achieved": vc_gbs64, "frac": vc_gbs64 / peak, "us": vc_us64}},
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
