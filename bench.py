"""Benchmark: PSFD solves/s to relative residual 1e-6 (warm vs cold) and matvec HBM GB/s.

One step = the whole hot path for one synthetic mask of the 128x128x64 workload
(2 nm pixels, random Manhattan layout of 4-24 rectangles, absorber n = 0.94+0.04i
with capping layer, TE + TM at 6 deg = 2 right-hand sides sharing one operator):
  mask -> smoothed fill (psfd_mask_fill) -> FP64 multilayer reflection and source
  b (psfd_background) -> factorised-FNO warm start for each polarisation
  (fno_forward, seed-initialised weights) -> spectral-damping right-preconditioned
  BiCGSTAB to ||b - A E|| / ||b|| <= 1e-6 (psfd_solve with x0) -> true residual.
`value` counts solved right-hand sides per second over the timed steps.  The same
step without the warm start (null initialisation) is reported as `cold`.

  python bench.py --gpus N --steps K --warmup W [--impl reference]

With --impl reference the FP64 CPU oracle (the test oracle of this repository) is
timed on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "manhattan_128x128x64"
TOL = 1e-6
PRACTICAL_TOL = 5e-2      # the paper's practical criterion (Sec. 3, Fig. 5a discussion)
MAXIT = 4000
BYTES_PER_POINT = 52.0   # algorithmic bytes of one A M apply per grid point and rhs


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--method", default="gmres", choices=["bicgstab", "gmres"])
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxit", type=int, default=MAXIT,
                    help="iteration cap per solve (lower it only for profiling runs)")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="run N HYBRID A M applies on one mask and exit (small ncu captures)")
    ap.add_argument("--nrhs", type=int, default=0, help="override the number of right-hand sides")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

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
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ----------------------------------------------------------------------------- GPU arm
def job_throughput(units_local: float, ms_local: float, world: int, device="cuda"):
    """Whole-job throughput across replicas: (units summed over ranks) / (max over ranks of the
    timed region).  Returns (units_total, ms_max).  world == 1: the local values."""
    if world <= 1:
        return units_local, ms_local
    import torch
    t = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    m = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(m, op=torch.distributed.ReduceOp.MAX)
    return float(t.item()), float(m.item())


def run_ours(args, rank, world):
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    prob = I.preset(args.workload)
    nrhs = args.nrhs or len(prob.pols)
    prob.pols = (prob.pols * nrhs)[:nrhs]
    stack = prob.stack()
    zprof = prob.zprofile()
    method = psfd.PSFD_GMRES if args.method == "gmres" else psfd.PSFD_BICGSTAB
    nsteps = args.warmup + args.steps
    tol_run = TOL
    # one seeded mask per step (rank-dependent seeds: independent problems per GPU)
    masks_host = [I.mask_for(prob, 1000 * rank + s) for s in range(nsteps)]
    masks = [torch.from_numpy(m).cuda() for m in masks_host]
    pinned = [torch.from_numpy(m).pin_memory() for m in masks_host]
    shape = I.FNOShape()
    models = []
    for pol in prob.pols:
        w = I.fno_weights(shape, 77 + pol)
        wd = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w.items()}
        models.append(psfd.fno_struct(wd, shape))
    plan = psfd.Plan(prob, nrhs=nrhs)
    ws = torch.empty(plan.workspace_size_ex(method, args.restart, True), dtype=torch.uint8, device="cuda")
    E = plan.empty()
    x0 = plan.empty()
    E_host = torch.empty(plan.shape, dtype=torch.complex64).pin_memory()
    stream = torch.cuda.current_stream()

    def step(i, warm=True, mask=None):
        fill = plan.mask_fill(masks[i] if mask is None else mask, zprof)
        b = plan.background(stack, fill, prob.pols)
        if warm:
            a = fill.unsqueeze(0).contiguous()
            for r, m in enumerate(models):
                psfd.fno_forward(m, a, out=x0[r:r + 1])
        res = plan.solve_ex(b, x0=x0 if warm else None, tol=tol_run, maxit=args.maxit, method=method,
                            restart=args.restart, refine=True, inner_tol=1e-2, out=E, workspace=ws)
        return res

    # warm-up (also exercises every kernel once)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    def timed(warm):
        infos = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = psfd.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, nsteps):
            infos.append(step(i, warm)["info"])
        e1.record(stream)
        torch.cuda.synchronize()
        launches = psfd.launch_count() - l0
        ms = e0.elapsed_time(e1)
        return ms, infos, launches

    clk = ClockSampler(dev)
    clk.start()
    ms_warm, info_warm, launches = timed(True)
    clocks = clk.stop()
    ms_cold, info_cold, _ = timed(False)
    # the same steps to the paper's practical criterion r_rel <= 5e-2
    tol_run = PRACTICAL_TOL
    ms_pw, info_pw, _ = timed(True)
    ms_pc, info_pc, _ = timed(False)
    tol_run = TOL

    # end to end through the public API: host mask in, host field out, copies inside the region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    info_e2e = []
    for i in range(args.warmup, nsteps):
        dm = pinned[i].to("cuda", non_blocking=True)
        info_e2e.append(step(i, True, mask=dm)["info"])
        E_host.copy_(E, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    h2d = pinned[0].numel() * pinned[0].element_size()
    d2h = E_host.numel() * E_host.element_size()

    # dominant operation: the A M matvec in the HYBRID domain, timed live with events
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    flags = psfd.PSFD_PRECOND | psfd.PSFD_HYBRID
    fill = plan.mask_fill(masks[0], zprof)
    plan.background(stack, fill, prob.pols)
    for _ in range(5):
        plan.apply(x, flags=flags, out=y)
    psfd.timing_enable(True)
    nap = 30
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(nap):
        plan.apply(x, flags=flags, out=y)
    eb.record(stream)
    torch.cuda.synchronize()
    stages = psfd.timing_read()
    psfd.timing_enable(False)
    ms_apply = ea.elapsed_time(eb) / nap
    # per-stage shares inside a warm solve step
    psfd.timing_enable(True)
    step(args.warmup, True)
    torch.cuda.synchronize()
    solve_stages = psfd.timing_read()
    psfd.timing_enable(False)

    npts = prob.nx * prob.ny * prob.nz * nrhs
    peak, peak_kind = measured_peaks()
    apply_bytes = npts * BYTES_PER_POINT
    # roofline of each stage inside the solve step: algorithmic bytes / CUDA-event time
    kernels = {"axial": "k_axial (fused M + stretched curl-curl + R column kernel)",
               "contrast": "k_rows/k_cols contrast passes (absorber planes)",
               "krylov": "Krylov vector kernels (k_vec, k_gdot, k_gupd, k_v64)",
               "transform": "lateral real<->HYBRID transforms (k_rows/k_cols)"}
    by_stage = {}
    for k, v in solve_stages.items():
        if v["calls"] and v["bytes"] > 0 and k in kernels:
            gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
            by_stage[k] = {"ms": v["ms"], "share": None, "GBps": gbs, "frac": gbs / peak,
                           "bytes_per_call": v["bytes"] / v["calls"], "ms_per_call": v["ms"] / v["calls"]}
    tot_ms = sum(v["ms"] for v in solve_stages.values() if v["calls"])
    for k in by_stage:
        by_stage[k]["share"] = by_stage[k]["ms"] / tot_ms
    dom = max(by_stage, key=lambda k: by_stage[k]["ms"])
    d = by_stage[dom]
    K = args.steps

    def converged(infos):
        return sum(1 for inf in infos for r in inf if r["status"] == 0)

    # only right-hand sides that reached the tolerance count as solves; units summed over the
    # replicas, time = the slowest replica's timed region
    def rate(infos, ms):
        units, ms_max = job_throughput(converged(infos), ms, world)
        return units / (ms_max / 1e3), ms_max

    value, ms_warm = rate(info_warm, ms_warm)
    cold_value, ms_cold = rate(info_cold, ms_cold)
    e2e_value, ms_e2e = rate(info_e2e, ms_e2e)
    pw_value, ms_pw = rate(info_pw, ms_pw)
    pc_value, ms_pc = rate(info_pc, ms_pc)
    iters_w = [r["iters"] for inf in info_warm for r in inf]
    iters_c = [r["iters"] for inf in info_cold for r in inf]
    rrel = [r["r_rel"] for inf in info_warm + info_cold for r in inf]
    status = [r["status"] for inf in info_warm + info_cold for r in inf]
    out = {
        "metric": "PSFD solves/s to rel. residual 1e-6 (warm start; cold alongside)",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_warm / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 (FP64 reductions, bf16 FNO mixing)",
        "data": "synthetic: seeded random Manhattan masks (4-24 rectangles, edges 4-40 px), "
                "seed-initialised FNO weights",
        "config": {"workload": args.workload, "grid": [prob.nx, prob.ny, prob.nz], "pixels_nm": [prob.dx, prob.dy, prob.dz],
                   "rhs_per_step": nrhs, "pols": ["TE", "TM"][:nrhs], "theta_deg": prob.theta_deg, "tol": TOL,
                   "solver": f"{args.method}({args.restart}) in complex64 with FP64 outer residual and field "
                             "(mixed-precision refinement, inner tol 1e-2), spectral-damping right preconditioner, "
                             "affine warm start",
                   "damping": {"m_min": prob.m_min, "gamma": prob.gamma, "k_ref": "k0"},
                   "l2": "working set (>= 9 vectors x 25 MB) exceeds the 126 MB L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "solve": {"iters_warm": iters_w, "iters_cold": iters_c, "r_rel_fp64_warm": [r["r_rel"] for inf in info_warm for r in inf],
                  "r_rel_fp64_cold": [r["r_rel"] for inf in info_cold for r in inf],
                  "r_rel_output_c64": [r["r_rel_output"] for inf in info_warm + info_cold for r in inf],
                  "status": status, "converged": f"{converged(info_warm) + converged(info_cold)} of {len(status)}",
                  "maxit": args.maxit, "outer_steps": [r["outer"] for inf in info_warm for r in inf],
                  "r_rel_initial_warm": [r["r_rel_initial"] for inf in info_warm for r in inf]},
        "cold": {"value": cold_value, "unit": "solves/s", "ms_per_step": ms_cold / K},
        "practical_5e-2": {"warm": {"value": pw_value, "ms_per_step": ms_pw / K,
                                    "iters": [r["iters"] for inf in info_pw for r in inf]},
                           "cold": {"value": pc_value, "ms_per_step": ms_pc / K,
                                    "iters": [r["iters"] for inf in info_pc for r in inf]},
                           "unit": "solves/s"},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "matvec": {"ms": ms_apply, "algorithmic_bytes": apply_bytes, "GBps_algorithmic": apply_bytes / ms_apply / 1e6,
                   "frac_of_peak": apply_bytes / ms_apply / 1e6 / peak, "stages_ms_per_apply":
                       {k: v["ms"] / nap for k, v in stages.items() if v["calls"]}},
        "roofline": {"kernel": kernels[dom], "stage": dom, "bound": "hbm", "achieved": d["GBps"], "peak": peak,
                     "unit": "GB/s", "frac": d["frac"], "traffic": None, "peak_kind": peak_kind,
                     "ms_per_launch": d["ms_per_call"], "algorithmic_bytes_per_launch": d["bytes_per_call"],
                     "share_of_step": d["share"]},
        "roofline_by_stage": by_stage,
        "solve_stage_ms": {k: v["ms"] for k, v in solve_stages.items() if v["calls"]},
        "clocks": clocks,
    }
    return out


def run_profile_apply(args):
    """N applies of A M in the HYBRID domain on one mask (for kernel captures)."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    prob = I.preset(args.workload)
    nrhs = args.nrhs or len(prob.pols)
    plan = psfd.Plan(prob, nrhs=nrhs)
    fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 0)).cuda(), prob.zprofile())
    plan.background(prob.stack(), fill, prob.pols[:nrhs] if nrhs <= len(prob.pols) else [0] * nrhs)
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.profile_apply):
        plan.apply(x, flags=psfd.PSFD_PRECOND | psfd.PSFD_HYBRID, out=y)
    e1.record()
    torch.cuda.synchronize()
    return {"profile_apply": args.profile_apply, "workload": args.workload, "nrhs": nrhs,
            "ms_per_apply": e0.elapsed_time(e1) / max(1, args.profile_apply)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(prob, seed, n_iter, method="gmres"):
    """Time the FP64 oracle: setup + a fixed number of Krylov iterations of the bench's method."""
    import torch
    from oracle import krylov as K
    from oracle import psfd as O
    from paper_2607_25330_b300 import inputs as I
    a = I.mask_for(prob, seed)
    t0 = time.perf_counter()
    g = O.Grid(prob.to_dict(), prob.stack())
    fill = O.fill_fraction(a, prob.zprofile(), prob.sigma_px)
    b = O.source_b(g, fill, prob.pols[0])
    t_setup = time.perf_counter() - t0
    A = lambda E: O.apply_A(g, E, fill)
    M = lambda x: O.apply_M(g, x)
    t1 = time.perf_counter()
    K.solve(A, M, b, tol=1e-30, maxit=n_iter, method=method, restart=30)
    t_it = (time.perf_counter() - t1) / n_iter
    return t_setup, t_it


def cpu_baseline(args, iters_per_solve):
    import torch
    from paper_2607_25330_b300 import inputs as I
    prob = I.preset(args.workload)
    n_iter = 6
    t_setup, t_it = oracle_sample(prob, 0, n_iter, args.method)
    s_per_solve = t_setup + t_it * iters_per_solve
    return {"value": 1.0 / s_per_solve, "unit": "solves/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle on one {args.workload} mask, one polarisation: setup + {n_iter} "
                      f"{args.method} iterations timed ({t_it:.2f} s/iteration, {t_setup:.2f} s setup), scaled to "
                      f"{iters_per_solve:.0f} iterations per solve (the GPU solve's mean count)"}


def run_reference(args):
    import torch
    from paper_2607_25330_b300 import inputs as I
    prob = I.preset(args.workload)
    iters_per_solve = float(MAXIT)   # the GPU arm's iteration cap per solve; stated, not measured here
    times = []
    for s in range(args.warmup + args.steps):
        t_setup, t_it = oracle_sample(prob, s, 2, args.method)
        if s >= args.warmup:
            times.append(t_setup + t_it * iters_per_solve)
    value = 1.0 / (sum(times) / len(times))
    cb = {"value": value, "unit": "solves/s", "cores": torch.get_num_threads(), "kind": "oracle",
          "sample": f"per step: FP64 oracle setup + 2 {args.method} iterations on one {args.workload} mask, "
                    f"scaled to {iters_per_solve:.0f} iterations per solve"}
    return {"impl": "reference", "metric": "PSFD solves/s to rel. residual 1e-6 (warm start; cold alongside)",
            "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.profile_apply:
        print(json.dumps(run_profile_apply(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            iters = out["solve"]["iters_warm"]
            out["cpu_baseline"] = cpu_baseline(args, float(np.mean(iters)) if iters else 1000.0)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
