"""Benchmark: PSFD solves/s to relative residual 1e-6 (warm vs cold) and matvec HBM GB/s.

One step = the whole hot path for one synthetic mask of the 128x128x64 workload
(2 nm pixels, random Manhattan layout of 4-24 rectangles, absorber n = 0.94+0.04i
with capping layer, TE + TM at 6 deg = 2 right-hand sides sharing one operator):
  mask -> smoothed fill (psfd_mask_fill) -> FP64 multilayer reflection and source
  b (psfd_background) -> layered-background preconditioner blocks (psfd_layered_build)
  -> factorised-FNO warm start for each polarisation (fno_forward, seed-initialised
  weights) -> right-preconditioned BiCGSTAB inside FP64 iterative refinement to
  ||b - A E|| / ||b|| <= 1e-6 (psfd_solve_ex with x0) -> FP64 true residual.
`value` counts solved right-hand sides per second over the timed steps.  The same
step without the warm start (null initialisation) is reported as `cold`; the
paper's own configurations (spectral damping M warm and cold, and no
preconditioner) run on the same masks under `paper_configurations`.

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
MAXIT = 600
BYTES_PER_POINT = 52.0   # algorithmic bytes of one A M apply per grid point and rhs


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--method", default="bicgstab", choices=["bicgstab", "gmres"],
                    help="inner Krylov method (BiCGSTAB is the paper's; GMRES(m) alongside)")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxit", type=int, default=MAXIT,
                    help="iteration cap per solve (lower it only for profiling runs)")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="run N HYBRID A M applies on one mask and exit (small ncu captures)")
    ap.add_argument("--profile-op", default="default", choices=["default", "A", "AM", "AP"],
                    help="operator of --profile-apply: A, A M, A P (default: A P with the layered P, else A M)")
    ap.add_argument("--profile-fno", type=int, default=0,
                    help="run N FNO forwards (B = 1) on the workload's grid and exit (small ncu captures)")
    ap.add_argument("--nrhs", type=int, default=0, help="override the number of right-hand sides")
    ap.add_argument("--precond", default="layered", choices=["layered", "damping"],
                    help="headline preconditioner: layered-background P (default) or the paper's damping M")
    ap.add_argument("--maxit-paper", type=int, default=12000,
                    help="iteration cap of the paper-configuration arms at 1e-6 and of the null arm")
    ap.add_argument("--paper-steps", type=int, default=2,
                    help="masks timed in each paper-configuration arm (its solves take seconds)")
    ap.add_argument("--maxit-bicgstab-paper", type=int, default=3000,
                    help="iteration cap of the arms with the paper's BiCGSTAB and damping M")
    ap.add_argument("--skip-paper-arms", action="store_true")
    ap.add_argument("--inner-tol", type=float, default=1e-3,
                    help="relative tolerance of each complex64 inner solve of the FP64 refinement")
    ap.add_argument("--train-step", action="store_true",
                    help="time the physics-informed FNO training step (16 masks 128x128x48) and exit")
    ap.add_argument("--train-batch", type=int, default=16)
    ap.add_argument("--skip-batch", action="store_true",
                    help="leave out the 384-rhs batching arm of the default run")
    ap.add_argument("--skip-fine", action="store_true",
                    help="leave out the 512x512x128 fine-discretisation arm of the default run")
    ap.add_argument("--skip-train-step", action="store_true",
                    help="leave out the timed physics-informed training step (16 masks 128x128x48) of the default run")
    ap.add_argument("--train-warm-steps", type=int, default=400,
                    help="Adam steps of the physics-informed training of the warm-start FNO (one model per "
                         "polarisation, on seeded masks disjoint from the timed ones) before the timed steps; "
                         "0 keeps the seed-initialised weights")
    ap.add_argument("--train-warm-batch", type=int, default=4)
    ap.add_argument("--lay-half", type=int, default=1,
                    help="store the layered blocks in half precision with per-block scales (1) or complex64 (0)")
    ap.add_argument("--lay-shift", type=float, default=0.25,
                    help="rebuild the layered blocks when a plane's mean fill moved by more than this")
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel from
# one ncu capture of the current kernel version on this workload (profiles/k_lay_apply_*.md):
# reported as roofline.traffic when the bench runs the same kernel on the same workload
NCU_TRAFFIC = {("precond", "manhattan_128x128x64", 2, True): 732.049664e6 + 46.290944e6}


def fp32_peak_tflops():
    """FP32 FMA peak of a B300 from its unit counts: 148 SMs x 128 lanes x 2 flop x 2.032 GHz."""
    return 148 * 128 * 2 * 2.032e9 / 1e12


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
    pc_main = psfd.PC_LAYERED if args.precond == "layered" else psfd.PC_DAMPING
    nsteps = args.warmup + args.steps
    # one seeded mask per step (rank-dependent seeds: independent problems per GPU)
    masks_host = [I.mask_for(prob, 1000 * rank + s) for s in range(nsteps)]
    masks = [torch.from_numpy(m).cuda() for m in masks_host]
    pinned = [torch.from_numpy(m).pin_memory() for m in masks_host]
    shape = I.FNOShape()
    models = []
    train_info = None
    if args.train_warm_steps > 0:
        # the warm start's network, trained here by the paper's physics loss (Sec. 3) with Adam:
        # one model per polarisation, on 32 seeded masks that the timed steps never see
        from paper_2607_25330_b300 import train as TR
        t_tr = time.perf_counter()
        train_info = {"steps": args.train_warm_steps, "batch": args.train_warm_batch, "pool": 32, "lr": 3e-3,
                      "output_layer": "zero-initialised (the untrained network predicts the cold start E = 0)",
                      "loss_first_last": []}
        for pol in prob.pols:
            w, log = TR.train(args.train_warm_steps, args.train_warm_batch, 3e-3, 32, 91 + pol, args.workload,
                              log_every=max(1, args.train_warm_steps // 4), pol=pol, mask_seed=50000 + 1000 * rank,
                              zero_output=True)
            wd = {k: v.detach().contiguous() for k, v in w.items()}
            models.append(psfd.fno_struct(wd, shape))
            train_info["loss_first_last"].append([log[0]["loss"], log[-1]["loss"]])
        torch.cuda.synchronize()
        train_info["seconds"] = time.perf_counter() - t_tr
    else:
        for pol in prob.pols:
            w = I.fno_weights(shape, 77 + pol)
            wd = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w.items()}
            models.append(psfd.fno_struct(wd, shape))
    plan = psfd.Plan(prob, nrhs=nrhs)
    if args.lay_half:
        plan.layered_storage(True)
    # sized for both methods: the paper-configuration arms run GMRES(30)
    ws_bytes = max(plan.workspace_size_ex(m, args.restart, True) for m in (psfd.PSFD_BICGSTAB, psfd.PSFD_GMRES))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    # the FP64 field is returned (complex128): its own residual is the one checked against 1e-6
    # (its complex64 rounding alone would carry about 1.3e-6 on this grid)
    E = torch.empty(plan.shape, dtype=torch.complex128, device="cuda")
    x0 = plan.empty()
    E_host = torch.empty(plan.shape, dtype=torch.complex128).pin_memory()
    stream = torch.cuda.current_stream()

    rebuilds = [0]

    def step(i, warm=True, mask=None, pc=pc_main, tol=TOL, maxit=args.maxit, rebuild="refresh", meth=None, out=None,
             itol=None):
        """The whole hot path for mask i: fill, background, preconditioner set-up, warm start, solve.

        The layered blocks depend on the mask only through each plane's mean fill; they are rebuilt
        when that moved by more than --lay-shift since the last build ("refresh"), or always."""
        fill = plan.mask_fill(masks[i] if mask is None else mask, zprof)
        b = plan.background(stack, fill, prob.pols)
        if pc == psfd.PC_LAYERED:
            if rebuild == "always":
                plan.layered_build()
                rebuilds[0] += 1
            elif plan.layered_refresh(args.lay_shift):
                rebuilds[0] += 1
        if warm:
            a = fill.unsqueeze(0).contiguous()
            for r, m in enumerate(models):
                psfd.fno_forward(m, a, out=x0[r:r + 1])
        return plan.solve_ex(b, x0=x0 if warm else None, tol=tol, maxit=maxit, method=method if meth is None else meth,
                             restart=args.restart, precond=pc, refine=True,
                             inner_tol=args.inner_tol if itol is None else itol,
                             out=E if out is None else out, workspace=ws, out_c128=True)

    # warm-up (also exercises every kernel once)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    def timed(count=None, **kw):
        """The steps of masks warmup .. warmup + count (all timed masks by default), CUDA events."""
        infos = []
        stop = nsteps if count is None else min(nsteps, args.warmup + count)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = psfd.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, stop):
            infos.append(step(i, **kw)["info"])
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), infos, psfd.launch_count() - l0

    def converged(infos):
        return sum(1 for inf in infos for r in inf if r["status"] == 0)

    # only right-hand sides that reached the tolerance count as solves; units summed over the
    # replicas, time = the slowest replica's timed region
    def rate(infos, ms):
        units, ms_max = job_throughput(converged(infos), ms, world)
        return units / (ms_max / 1e3), ms_max

    def arm(t):
        ms, infos, _ = t
        v, msm = rate(infos, ms)
        return {"value": v, "ms_per_step": msm / max(1, len(infos)), "masks": len(infos),
                "converged": f"{converged(infos)} of {sum(len(x) for x in infos)}",
                "iters": [r["iters"] for inf in infos for r in inf],
                "r_rel_fp64": [r["r_rel"] for inf in infos for r in inf],
                "r_rel_initial": [r["r_rel_initial"] for inf in infos for r in inf]}

    # clocks are sampled over all timed arms (the headline arm alone lasts well under a second)
    clk = ClockSampler(dev)
    clk.start()
    rebuilds[0] = 0
    ms_warm, info_warm, launches = timed(warm=True)
    rebuilds_warm = rebuilds[0]
    ms_cold, info_cold, _ = timed(warm=False)
    # the same warm steps with the blocks rebuilt for every mask (no reuse across masks)
    layered_always = None
    if pc_main == psfd.PC_LAYERED:
        layered_always = arm(timed(warm=True, rebuild="always"))

    # end to end through the public API: host mask in, host field out, every step's copies inside
    # the region. The field of step k goes to the host on a copy stream while step k + 1 computes
    # (two device fields and two pinned host buffers; a step waits for the copy that last used its
    # buffers), and the region ends when the last copy has landed.
    torch.cuda.synchronize()
    copy_stream = torch.cuda.Stream()
    E_bufs = [E, torch.empty_like(E)]
    E_hosts = [E_host, torch.empty(plan.shape, dtype=torch.complex128).pin_memory()]
    copied = [None, None]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    info_e2e = []
    for k, i in enumerate(range(args.warmup, nsteps)):
        j = k % 2
        dm = pinned[i].to("cuda", non_blocking=True)
        if copied[j] is not None:
            stream.wait_event(copied[j])
        info_e2e.append(step(i, True, mask=dm, out=E_bufs[j])["info"])
        ready = torch.cuda.Event()
        ready.record(stream)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            E_hosts[j].copy_(E_bufs[j], non_blocking=True)
            copied[j] = torch.cuda.Event()
            copied[j].record(copy_stream)
    stream.wait_stream(copy_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    h2d = pinned[0].numel() * pinned[0].element_size()
    d2h = E_host.numel() * E_host.element_size()

    # the paper's configurations on the same masks: spectral damping M (warm, cold) and the null
    # configuration (no preconditioner, cold), at 1e-6 and at the practical 5e-2, each on
    # --paper-steps masks (their solves take seconds)
    paper = {}
    if not args.skip_paper_arms:
        pd, gm, bi = psfd.PC_DAMPING, psfd.PSFD_GMRES, psfd.PSFD_BICGSTAB
        n_p, mp, mb = args.paper_steps, args.maxit_paper, args.maxit_bicgstab_paper
        paper["damping_gmres30_warm_1e-6"] = arm(timed(n_p, warm=True, pc=pd, maxit=mp, meth=gm, itol=1e-2))
        paper["damping_gmres30_cold_1e-6"] = arm(timed(n_p, warm=False, pc=pd, maxit=mp, meth=gm, itol=1e-2))
        paper["damping_bicgstab_warm_1e-6"] = arm(timed(n_p, warm=True, pc=pd, maxit=mb, meth=bi, itol=1e-2))
        paper["damping_bicgstab_cold_1e-6"] = arm(timed(n_p, warm=False, pc=pd, maxit=mb, meth=bi, itol=1e-2))
        paper["damping_gmres30_warm_5e-2"] = arm(timed(n_p, warm=True, pc=pd, tol=PRACTICAL_TOL, maxit=mp, meth=gm))
        paper["damping_gmres30_cold_5e-2"] = arm(timed(n_p, warm=False, pc=pd, tol=PRACTICAL_TOL, maxit=mp, meth=gm))
        paper["null_gmres30_cold_5e-2"] = arm(timed(n_p, warm=False, pc=psfd.PC_NONE, tol=PRACTICAL_TOL, maxit=mp,
                                                    meth=gm))
        for k, mx in (("damping_bicgstab_warm_1e-6", mb), ("damping_bicgstab_cold_1e-6", mb)):
            paper[k]["maxit"] = mx
        for k in paper:
            paper[k].setdefault("maxit", mp)
        # the paper's own illumination, normal incidence (its runs are TE at 0 deg), cold start
        prob0 = I.preset(args.workload)
        prob0.theta_deg = 0.0
        prob0.pols = list(prob.pols)
        plan0 = psfd.Plan(prob0, nrhs=nrhs)
        ms0, inf0 = 0.0, []
        torch.cuda.synchronize()
        for i in range(args.warmup, min(nsteps, args.warmup + n_p)):
            fill0 = plan0.mask_fill(masks[i], zprof)
            b0_ = plan0.background(stack, fill0, prob0.pols)
            e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0_.record(stream)
            r0_ = plan0.solve_ex(b0_, tol=TOL, maxit=mp, method=gm, restart=args.restart, precond=pd, refine=True,
                                 inner_tol=1e-2, out_c128=True, workspace=ws)
            e1_.record(stream)
            torch.cuda.synchronize()
            ms0 += e0_.elapsed_time(e1_)
            inf0.append(r0_["info"])
        paper["damping_gmres30_cold_1e-6_theta0"] = arm((ms0, inf0, 0))
        paper["damping_gmres30_cold_1e-6_theta0"]["maxit"] = mp
        plan0.close()
        del plan0
        paper["note"] = ("the paper's spectral damping M (Eqs. spectral_damping_action, spectral_damping_mask) and "
                         "null configuration on the same masks, in the same FP64 refinement: GMRES(30) inner "
                         "solves, and the paper's BiCGSTAB (which diverges in complex64 on this operator); "
                         "only right-hand sides that reached the tolerance within maxit count; theta0: the "
                         "paper's normal incidence")

    # the paper's practical criterion (Sec. 4): iterations until the threshold-contour widths of
    # |E_y|^2 on the plane above the absorber are within 1 nm (wafer units, /4) of the converged
    # field's, on one mask, rhs 0 (TE)
    width = {}
    if not args.skip_paper_arms:
        i0 = args.warmup
        fill = plan.mask_fill(masks[i0], zprof)
        b0 = plan.background(stack, fill, prob.pols)
        if pc_main == psfd.PC_LAYERED:
            plan.layered_build()
        a0 = fill.unsqueeze(0).contiguous()
        for r, m in enumerate(models):
            psfd.fno_forward(m, a0, out=x0[r:r + 1])
        ref = plan.solve_ex(b0, tol=1e-7, maxit=args.maxit, precond=pc_main)["E"].clone()   # complex64
        zp = np.asarray(zprof)
        ztop = int(np.nonzero(zp > 0)[0].max()) + 1
        grids = {"layered": [1, 2, 3, 4, 6, 8, 12, 16, 24, 32], "damping": [10, 20, 40, 80, 160, 320, 640]}
        for name, pc in (("layered", psfd.PC_LAYERED), ("damping", psfd.PC_DAMPING)):
            if name == "layered" and pc_main != psfd.PC_LAYERED:
                continue
            for warm in (True, False):
                hit, trace = None, []
                for k in grids[name]:
                    E_k = plan.solve(b0, x0=x0 if warm else None, tol=1e-12, maxit=k,
                                     method=method if pc == psfd.PC_LAYERED else psfd.PSFD_GMRES,
                                     restart=args.restart, precond=pc)["E"]
                    mtr = plan.width_metric(E_k, ref, ztop, rhs=0, comp=1, I_th=0.15, n_lines=100, demag=4.0)
                    trace.append([k, round(mtr["mean"], 4), mtr["matched"], mtr["unresolved"]])
                    if hit is None and mtr["matched"] > 0 and mtr["mean"] <= 1.0:
                        hit = k
                        break
                width[f"{name}_{'warm' if warm else 'cold'}"] = {"iters_to_mean_below_1nm": hit, "trace": trace}
        width["definition"] = ("I = |E_y|^2 on the first plane above the absorber, I_th = 0.15, 100 + 100 scan "
                               "lines, widths of threshold-bounded segments, |d_ref - d| / 4 against the 1e-7 "
                               "solution; criterion: mean <= 1 nm (the paper's sub-nanometre level); "
                               "trace = [iterations, mean nm, matched, unresolved reference segments]")

    clocks = clk.stop()
    clocks["window"] = "all timed arms (headline, cold, e2e, rebuild-every-mask, paper configurations)"

    # per-stage CUDA-event timing inside one headline step (stage byte counts are algorithmic)
    psfd.timing_enable(True)
    step(args.warmup, True)
    torch.cuda.synchronize()
    solve_stages = psfd.timing_read()
    psfd.timing_enable(False)

    build_stages = None
    if pc_main == psfd.PC_LAYERED:
        psfd.timing_enable(True)
        plan.layered_build()
        torch.cuda.synchronize()
        build_stages = psfd.timing_read()
        psfd.timing_enable(False)

    # dominant operations timed live: the A P matvec pieces in the HYBRID domain
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    nap = 20
    psfd.timing_enable(True)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(nap):
        plan.apply(x, flags=psfd.PSFD_HYBRID | (psfd.PSFD_LAYERED if pc_main == psfd.PC_LAYERED else psfd.PSFD_PRECOND),
                   out=y)
    eb.record(stream)
    torch.cuda.synchronize()
    mv_stages = psfd.timing_read()
    psfd.timing_enable(False)
    ms_apply = ea.elapsed_time(eb) / nap
    # the paper's operator alone: y = A x in the HYBRID domain (the Krylov vectors' domain)
    psfd.timing_enable(True)
    ea.record(stream)
    for _ in range(nap):
        plan.apply(x, flags=psfd.PSFD_HYBRID, out=y)
    eb.record(stream)
    torch.cuda.synchronize()
    a_stages = psfd.timing_read()
    psfd.timing_enable(False)
    ms_A = ea.elapsed_time(eb) / nap

    npts = prob.nx * prob.ny * prob.nz * nrhs
    peak, peak_kind = measured_peaks()
    fp32_peak = fp32_peak_tflops()
    # Gauss-Jordan inversion of the TE (nz) and TM (2 nz) blocks of every lateral column:
    # N^3 complex multiply-adds (8 real flops each) per N x N block
    # (ky and -ky share their blocks when there is no Bloch shift along y: ny/2 + 1 stored rows)
    lay_rows = prob.ny // 2 + 1 if (prob.phi_deg == 0.0 or prob.theta_deg == 0.0) and prob.ny % 2 == 0 else prob.ny
    lay_flops = prob.nx * lay_rows * 8.0 * (prob.nz ** 3 + (2 * prob.nz) ** 3)
    kernels = {"axial": "k_axial (fused curl-curl + R column kernel)",
               "contrast": "k_rows/k_cols contrast passes (absorber planes)",
               "krylov": "Krylov vector kernels (k_vec, k_gdot, k_gupd, k_v64)",
               "transform": "lateral real<->HYBRID transforms (k_rows/k_cols)",
               "precond": "k_lay_apply_pipe (per-column TE/TM inverse blocks x vectors, tensor cores)",
               "lay_build": "k_lay_inv (per-column TE/TM assembly + Gauss-Jordan inversion, FP32)",
               "fno": "FNO forward kernels"}
    by_stage = {}
    tot_ms = sum(v["ms"] for v in solve_stages.values() if v["calls"])
    for k, v in solve_stages.items():
        if not v["calls"] or k not in kernels:
            continue
        e = {"ms": v["ms"], "share": v["ms"] / tot_ms, "calls": v["calls"], "ms_per_call": v["ms"] / v["calls"]}
        if k == "lay_build":
            tf = lay_flops / (v["ms"] / v["calls"] / 1e3) / 1e12
            e.update({"bound": "alu", "TFLOPs_fp32": tf, "frac": tf / fp32_peak,
                      "flops_per_call": lay_flops})
        elif v["bytes"] > 0:
            # the operator and preconditioner kernels skip right-hand sides that have converged, so
            # inside the solve their stage counts bytes for launches that did no work: their rate
            # comes from the dedicated A P applies above (every right-hand side active)
            src = v
            if k in ("axial", "contrast", "precond") and mv_stages.get(k, {}).get("calls"):
                src = mv_stages[k]
            gbs = src["bytes"] / (src["ms"] / 1e3) / 1e9
            e.update({"bound": "hbm", "GBps": gbs, "frac": gbs / peak, "bytes_per_call": src["bytes"] / src["calls"],
                      "ms_per_launch": src["ms"] / src["calls"],
                      "rate_from": "dedicated applies" if src is not v else "inside the solve"})
        by_stage[k] = e
    if build_stages is not None and build_stages["lay_build"]["calls"]:
        v = build_stages["lay_build"]
        tf = lay_flops / (v["ms"] / v["calls"] / 1e3) / 1e12
        by_stage.setdefault("lay_build", {"ms": v["ms"], "share": 0.0, "calls": v["calls"],
                                          "ms_per_call": v["ms"] / v["calls"], "bound": "alu",
                                          "TFLOPs_fp32": tf, "frac": tf / fp32_peak, "flops_per_call": lay_flops,
                                          "note": "timed on a separate rebuild: the headline step reused the blocks"})
    # the roofline is the dominant single kernel's: among stages with algorithmic bytes or flops
    # that are one kernel (the preconditioner apply); the Krylov stage is five vector kernels, the
    # axial and contrast stages several, and the FNO stage has no byte count (all are reported by
    # their time in roofline_by_stage)
    single = [k for k in ("precond", "axial") if "bound" in by_stage.get(k, {}) and by_stage[k]["share"] > 0]
    dom = max(single, key=lambda k: by_stage[k]["share"]) if single else \
        max((k for k in by_stage if "bound" in by_stage[k]), key=lambda k: by_stage[k]["ms"] * (by_stage[k]["share"] > 0))
    d = by_stage[dom]
    if d.get("bound") == "alu":
        roof = {"kernel": kernels[dom], "stage": dom, "bound": "alu", "achieved": d["TFLOPs_fp32"],
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": d["frac"], "traffic": None,
                "peak_kind": "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz",
                "ms_per_launch": d["ms_per_call"], "algorithmic_flops_per_launch": lay_flops,
                "share_of_step": d["share"]}
    else:
        traffic = NCU_TRAFFIC.get((dom, args.workload, nrhs, bool(args.lay_half)))
        roof = {"kernel": kernels[dom], "stage": dom, "bound": "hbm", "achieved": d["GBps"], "peak": peak,
                "unit": "GB/s", "frac": d["frac"], "traffic": traffic, "peak_kind": peak_kind,
                "traffic_source": "ncu capture in profiles/ (dram read + write per launch)" if traffic else None,
                "ms_per_launch": d.get("ms_per_launch", d["ms_per_call"]), "algorithmic_bytes_per_launch": d["bytes_per_call"],
                "share_of_step": d["share"]}
    K = args.steps
    value, ms_warm_max = rate(info_warm, ms_warm)
    cold_value, ms_cold_max = rate(info_cold, ms_cold)
    e2e_value, _ = rate(info_e2e, ms_e2e)
    pc_name = {psfd.PC_LAYERED: "layered-background preconditioner P (per-mode TE/TM inverse of the "
                                "laterally averaged operator; not in the paper)",
               psfd.PC_DAMPING: "spectral damping M (the paper's preconditioner)"}[pc_main]
    out = {
        "metric": "PSFD solves/s to rel. residual 1e-6 (warm start; cold alongside)",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_warm_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 (Krylov, operator, preconditioner; FP64 reductions, refinement residual and returned field; "
                 "bf16 FNO mixing)",
        "data": "synthetic: seeded random Manhattan masks (4-24 rectangles, edges 4-40 px); " +
                (f"warm-start FNO trained in this run by the physics loss ({args.train_warm_steps} Adam steps per "
                 "polarisation on 32 seeded masks disjoint from the timed ones, outside the timed region)"
                 if args.train_warm_steps > 0 else "seed-initialised FNO weights"),
        "warm_start_training": train_info,
        "config": {"workload": args.workload, "grid": [prob.nx, prob.ny, prob.nz], "pixels_nm": [prob.dx, prob.dy, prob.dz],
                   "rhs_per_step": nrhs, "pols": ["TE", "TM"][:nrhs], "theta_deg": prob.theta_deg, "tol": TOL,
                   "preconditioner": pc_name,
                   "preconditioner_setup": (f"per-mask refresh: blocks rebuilt only when a plane's mean fill moved by "
                                            f"> {args.lay_shift} since the last build; {rebuilds_warm} rebuilds in the "
                                            "timed warm steps (rebuilding for every mask: "
                                            "layered_blocks.warm_with_rebuild_every_mask)")
                                           if pc_main == psfd.PC_LAYERED else "none (M is a fixed multiplier)",
                   "solver": (f"{args.method}({args.restart})" if args.method == "gmres" else args.method) +
                             " in complex64 inside FP64 iterative refinement "
                             f"(FP64 residual and field, inner tol {args.inner_tol:g}), right preconditioning, "
                             "affine warm start",
                   "step": "mask -> fill -> FP64 TMM + source -> preconditioner set-up -> FNO warm start -> "
                           "solve -> FP64 true residual",
                   "l2": "working set (2.7 GB of blocks + >= 9 vectors x 25 MB) exceeds the 126 MB L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "solve": {"iters_warm": [r["iters"] for inf in info_warm for r in inf],
                  "iters_cold": [r["iters"] for inf in info_cold for r in inf],
                  "outer_steps_warm": [r["outer"] for inf in info_warm for r in inf],
                  "r_rel_fp64_warm": [r["r_rel"] for inf in info_warm for r in inf],
                  "r_rel_fp64_cold": [r["r_rel"] for inf in info_cold for r in inf],
                  "r_rel_output_field": [r["r_rel_output"] for inf in info_warm + info_cold for r in inf],
                  "output": "FP64 field (complex128)",
                  "r_rel_initial_warm": [r["r_rel_initial"] for inf in info_warm for r in inf],
                  "converged": f"{converged(info_warm) + converged(info_cold)} of "
                               f"{sum(len(x) for x in info_warm + info_cold)}", "maxit": args.maxit},
        "cold": {"value": cold_value, "unit": "solves/s", "ms_per_step": ms_cold_max / K},
        "layered_blocks": {"reuse_rule": f"rebuilt when a plane's mean fill moved by > {args.lay_shift} "
                                         "since the last build (psfd_layered_refresh)",
                           "storage": "half precision, power-of-two scale per block" if args.lay_half else "complex64",
                           "bytes": plan.layered_bytes(),
                           "rebuilds_in_timed_warm_steps": rebuilds_warm,
                           "warm_with_rebuild_every_mask": layered_always},
        "paper_configurations": paper,
        "practical_width_criterion": width,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "matvec": {"ms_per_A_P_apply": ms_apply, "stages_ms_per_apply":
                   {k: v["ms"] / nap for k, v in mv_stages.items() if v["calls"]},
                   "GBps_algorithmic": {k: v["bytes"] / (v["ms"] / 1e3) / 1e9 for k, v in mv_stages.items()
                                        if v["calls"] and v["bytes"] > 0},
                   "A_bytes_per_point_rhs": BYTES_PER_POINT, "points_x_rhs": npts},
        "roofline": roof,
        "roofline_matvec": {
            "kernel": "A apply of the paper's operator, HYBRID domain: k_axial (curl-curl, PML, R) + lateral "
                      "contrast passes (k_rows, k_cols)",
            "bound": "hbm", "achieved": BYTES_PER_POINT * npts / (ms_A / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": BYTES_PER_POINT * npts / (ms_A / 1e3) / 1e9 / peak,
            "frac_of_8TBps_spec": BYTES_PER_POINT * npts / (ms_A / 1e3) / 1e9 / 8000.0,
            "ms_per_apply": ms_A, "algorithmic_bytes_per_apply": BYTES_PER_POINT * npts,
            "algorithmic": f"{BYTES_PER_POINT:g} B per point and rhs (read 24, write 24, deps 4) x {npts} points x rhs",
            "stages_ms_per_apply": {k: v["ms"] / nap for k, v in a_stages.items() if v["calls"]},
            "stage_GBps_own_bytes": {k: v["bytes"] / (v["ms"] / 1e3) / 1e9 for k, v in a_stages.items()
                                     if v["calls"] and v["bytes"] > 0},
            "peak_kind": peak_kind},
        "roofline_by_stage": by_stage,
        "solve_stage_ms": {k: v["ms"] for k, v in solve_stages.items() if v["calls"]},
        "clocks": clocks,
    }
    return out


def run_fine(args):
    """The fine-discretisation workload at full size: 512x512x128 (0.5 nm lateral pixels), TE + TM at
    6 deg, a dense Manhattan layout; warm start from the FNO evaluated on the 128x128x128 grid of the
    same box and axial planes (2 nm lateral pixels) and spectrally upsampled in x and y (the network
    trained on that coarse grid by the physics loss, on dense layouts of the same recipe),
    against the cold start; GMRES(30) in complex64 with FP64 orthogonalisation inside the FP64
    refinement, layered-background P (Schur form at nz = 128), to 1e-6.  Also the A apply's roofline
    at this size, where the vectors (0.8 GB per rhs) are far larger than L2."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    prob = I.preset("fine_512x512x128")
    coarse = I.preset("fno_coarse_128x128x128")
    shape = I.FNOShape()
    out = {"workload": "fine_512x512x128", "grid": [prob.nx, prob.ny, prob.nz], "pixels_nm": [prob.dx, prob.dy, prob.dz],
           "coarse_grid": [coarse.nx, coarse.ny, coarse.nz], "solver": "gmres(30), FP64 refinement (inner 1e-3)",
           "preconditioner": "layered-background P, Schur form, complex64 blocks", "tol": TOL}
    models = []
    t0 = time.perf_counter()
    if args.train_warm_steps > 0:
        from paper_2607_25330_b300 import train as TR
        for pol in prob.pols:
            w, log = TR.train(max(1, args.train_warm_steps // 2), args.train_warm_batch, 3e-3, 32, 191 + pol,
                              "fno_coarse_128x128x128", log_every=max(1, args.train_warm_steps // 4), pol=pol,
                              mask_seed=70000, zero_output=True, mask_kind="manhattan_dense")
            models.append(psfd.fno_struct({k: v.detach().contiguous() for k, v in w.items()}, shape))
        out["coarse_training"] = {"steps": max(1, args.train_warm_steps // 2), "seconds": time.perf_counter() - t0}
    else:
        for pol in prob.pols:
            w = I.fno_weights(shape, 77 + pol)
            models.append(psfd.fno_struct({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w.items()},
                                          shape))
    plan = psfd.Plan(prob)
    plan.layered_storage(True)
    cplan = psfd.Plan(coarse, nrhs=1)
    ws = torch.empty(plan.workspace_size_ex(psfd.PSFD_GMRES, 30, True), dtype=torch.uint8, device="cuda")
    E = torch.empty(plan.shape, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for warm in (True, False):
        infos, ms = [], 0.0
        for k in range(2):
            a = I.mask_for(prob, 400 + k, "manhattan_dense")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fill = plan.mask_fill(torch.from_numpy(a).cuda(), prob.zprofile())
            b = plan.background(prob.stack(), fill, prob.pols)
            plan.layered_build()
            x0 = None
            if warm:
                cfill = cplan.mask_fill(torch.from_numpy(np.ascontiguousarray(a[::4, ::4])).cuda(), coarse.zprofile())
                Ec = torch.cat([psfd.fno_forward(m, cfill[None].contiguous()) for m in models])
                x0 = psfd.spectral_upsample(Ec, prob.nz, prob.ny, prob.nx).contiguous()
            r = plan.solve_ex(b, x0=x0, tol=TOL, maxit=2000, method=psfd.PSFD_GMRES, restart=30,
                              precond=psfd.PC_LAYERED, inner_tol=1e-3, out=E, workspace=ws, out_c128=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            infos.append(r["info"])
        conv = sum(1 for inf in infos for i in inf if i["status"] == 0)
        res["warm" if warm else "cold"] = {
            "value": conv / (ms / 1e3), "unit": "solves/s", "ms_per_mask": ms / len(infos),
            "converged": f"{conv} of {sum(len(x) for x in infos)}",
            "iters": [i["iters"] for inf in infos for i in inf], "r_rel_fp64": [i["r_rel"] for inf in infos for i in inf],
            "r_rel_initial": [i["r_rel_initial"] for inf in infos for i in inf],
            "step": "mask -> fill -> TMM + source -> P build -> (coarse FNO + upsample) -> solve, all timed"}
    out.update(res)
    # the A apply at this size (HBM-bound), CUDA events on the launching stream
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    nap = 5
    plan.apply(x, flags=psfd.PSFD_HYBRID, out=y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    psfd.timing_enable(True)
    e0.record(stream)
    for _ in range(nap):
        plan.apply(x, flags=psfd.PSFD_HYBRID, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    st = psfd.timing_read()
    psfd.timing_enable(False)
    ms_A = e0.elapsed_time(e1) / nap
    npts = prob.nx * prob.ny * prob.nz * len(prob.pols)
    peak, peak_kind = measured_peaks()
    gbs = BYTES_PER_POINT * npts / (ms_A / 1e3) / 1e9
    out["roofline_matvec"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                              "frac_of_8TBps_spec": gbs / 8000.0, "ms_per_apply": ms_A,
                              "algorithmic_bytes_per_apply": BYTES_PER_POINT * npts,
                              "stages_ms_per_apply": {k: v["ms"] / nap for k, v in st.items() if v["calls"]},
                              "stage_GBps_own_bytes": {k: v["bytes"] / (v["ms"] / 1e3) / 1e9 for k, v in st.items()
                                                       if v["calls"] and v["bytes"] > 0},
                              "peak_kind": peak_kind}
    out["layered_bytes"] = plan.layered_bytes()
    plan.close()
    cplan.close()
    return out


def run_batch(args, chunk=16):
    """The batching workload at its size: 64 Manhattan masks of uneven lateral size (64^2, 96^2,
    128^2, 256^2) and depth (nz 32, 48, 64, 96), each at 3 angles (4, 6, 8 deg) x TE + TM = 384
    right-hand sides, 192 operators.  Per chunk of operators: plans on their own streams, fill,
    TMM + source, layered P (Schur form for nz 32, 64 and 96: each operator's blocks serve one solve
    and the Schur build is about 3x cheaper; half-precision full blocks at nz 48), then psfd_solve_batched
    (BiCGSTAB in FP64 refinement to 1e-6) over the chunk on concurrent streams; plans freed per
    chunk.  Everything from the device-resident mask to the FP64 residual is timed (host clock
    around the whole set; one device synchronisation per chunk)."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    probs = I.batch_presets()
    # the seeded layouts are the inputs: generated and resident on the device before the clock starts,
    # as in the headline workload
    dmasks = [torch.from_numpy(I.mask_for(pr, 600 + idx // 3)).cuda() for idx, pr in enumerate(probs)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos_all, by_size = [], {}
    for c0 in range(0, len(probs), chunk):
        group = probs[c0:c0 + chunk]
        streams = [torch.cuda.Stream() for _ in group]
        plans, bs = [], []
        for k, (pr, st) in enumerate(zip(group, streams)):
            idx = c0 + k                                 # one mask per 3 angles
            pl = psfd.Plan(pr, stream=st)
            pl.layered_storage(True)
            pl.layered_form(True)      # blocks built for one solve: the cheaper Schur build
            with torch.cuda.stream(st):
                fill = pl.mask_fill(dmasks[idx], pr.zprofile())
                b = pl.background(pr.stack(), fill, pr.pols)
            pl.layered_build()
            plans.append(pl)
            bs.append(b)
        torch.cuda.synchronize()
        Es, infos = psfd.solve_batched(plans, bs, tol=TOL, maxit=600, method=psfd.PSFD_BICGSTAB, precond=2,
                                       refine=True, inner_tol=1e-3, nworkers=8)
        for pr, inf in zip(group, infos):
            key = f"{pr.nx}x{pr.ny}x{pr.nz}"
            d = by_size.setdefault(key, {"rhs": 0, "converged": 0, "iters": []})
            d["rhs"] += len(inf)
            d["converged"] += sum(1 for i in inf if i["status"] == 0)
            d["iters"] += [i["iters"] for i in inf]
        infos_all += infos
        del Es, bs
        for pl in plans:
            pl.close()
        torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    conv = sum(1 for inf in infos_all for i in inf if i["status"] == 0)
    total = sum(len(inf) for inf in infos_all)
    for d in by_size.values():
        d["mean_iters"] = float(np.mean(d["iters"])) if d["iters"] else None
        del d["iters"]
    return {"workload": "batch_64_masks_x_3_angles_x_2_pols", "operators": len(probs), "rhs": total,
            "converged": f"{conv} of {total}", "seconds": sec, "value": conv / sec, "unit": "solves/s",
            "points_all_rhs": int(sum(p.nx * p.ny * p.nz * len(p.pols) for p in probs)),
            "by_grid": by_size, "max_r_rel_fp64": max(i["r_rel"] for inf in infos_all for i in inf),
            "execution": f"chunks of {chunk} operators on their own streams, psfd_solve_batched with 8 host "
                         "workers (concurrent streams; not one persistent launch)"}


def run_profile_apply(args):
    """N applies of A P (layered) or A M (damping) in the HYBRID domain on one mask (kernel captures)."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    prob = I.preset(args.workload)
    nrhs = args.nrhs or len(prob.pols)
    plan = psfd.Plan(prob, nrhs=nrhs)
    fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 0)).cuda(), prob.zprofile())
    plan.background(prob.stack(), fill, prob.pols[:nrhs] if nrhs <= len(prob.pols) else [0] * nrhs)
    flags = psfd.PSFD_HYBRID | psfd.PSFD_PRECOND
    if args.profile_op in ("default", "AP") and args.precond == "layered" and plan.layered_bytes() > 0:
        if args.lay_half:
            plan.layered_storage(True)
        plan.layered_build()
        flags = psfd.PSFD_HYBRID | psfd.PSFD_LAYERED
    elif args.profile_op == "A":
        flags = psfd.PSFD_HYBRID
    x = torch.randn(plan.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.profile_apply):
        plan.apply(x, flags=flags, out=y)
    e1.record()
    torch.cuda.synchronize()
    return {"profile_apply": args.profile_apply, "workload": args.workload, "nrhs": nrhs, "flags": flags,
            "ms_per_apply": e0.elapsed_time(e1) / max(1, args.profile_apply)}


def run_profile_fno(args):
    """N forwards of the seed-initialised FNO (B = 1) on the workload's grid (kernel captures)."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    prob = I.preset(args.workload)
    S = I.FNOShape()
    w = I.fno_weights(S, 77)
    ws = psfd.fno_struct({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w.items()}, S)
    a = torch.rand((1, prob.nz, prob.ny, prob.nx), device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    out = torch.empty((1, 3, prob.nz, prob.ny, prob.nx), dtype=torch.complex64, device="cuda")
    for _ in range(3):
        psfd.fno_forward(ws, a, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.profile_fno):
        psfd.fno_forward(ws, a, out=out)
    e1.record()
    torch.cuda.synchronize()
    return {"profile_fno": args.profile_fno, "workload": args.workload,
            "ms_per_forward": e0.elapsed_time(e1) / max(1, args.profile_fno)}


def run_train_step(args, steps=None, warmup=None):
    """Physics-informed training step of the factorised FNO (config 4): 16 masks 128x128x48,
    E = G_theta(a) for the batch, J = mean over masks of Eq. loss through the PSFD operator
    (hand-written adjoint), reverse pass of the FNO (checkpointed), Adam update."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    from paper_2607_25330_b300 import psfd
    from paper_2607_25330_b300.autograd import fno_apply, physics_loss
    prob = I.preset("fno_train_128x128x48")
    B = args.train_batch
    S = I.FNOShape()
    w = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().requires_grad_(True)
         for k, v in I.fno_weights(S, 91, spectral_scale=1.0).items()}
    trainer = psfd.FnoTrainer(psfd.fno_struct(w, S), B, prob.nz, prob.ny, prob.nx, checkpoint=True)
    plans, bs, fills = [], [], []
    for s in range(B):
        pl = psfd.Plan(prob, nrhs=1)
        fill = pl.mask_fill(torch.from_numpy(I.mask_for(prob, 500 + s)), prob.zprofile())
        bs.append(pl.background(prob.stack(), fill, prob.pols))
        plans.append(pl)
        fills.append(fill)
    a = torch.stack(fills).contiguous()
    opt = torch.optim.Adam(list(w.values()), lr=1e-3)

    def train_step():
        opt.zero_grad(set_to_none=True)
        E = fno_apply(trainer, w, a)
        J = sum(physics_loss(plans[s], E[s:s + 1], bs[s]) for s in range(B)) / B
        J.backward()
        opt.step()
        return J

    n_steps = args.steps if steps is None else steps
    n_warm = args.warmup if warmup is None else warmup
    for _ in range(n_warm):
        train_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    psfd.timing_enable(True)
    e0.record()
    losses = [train_step() for _ in range(n_steps)]
    e1.record()
    torch.cuda.synchronize()
    st = psfd.timing_read()
    psfd.timing_enable(False)
    ms = e0.elapsed_time(e1) / n_steps
    mem = torch.cuda.max_memory_allocated() / 2 ** 30
    return {"mode": "train_step", "workload": "fno_train_128x128x48", "batch": B, "steps": n_steps,
            "warmup": n_warm, "ms_per_step": ms, "masks_per_s": B / (ms / 1e3),
            "loss": [float(l) for l in losses], "fno_ms_per_step": st["fno"]["ms"] / n_steps,
            "psfd_ms_per_step": (st["axial"]["ms"] + st["contrast"]["ms"]) / n_steps,
            "workspace_GiB": trainer.n / 2 ** 30, "max_allocated_GiB": mem,
            "note": "forward + physics loss (PSFD apply and adjoint per mask) + checkpointed FNO reverse pass + "
                    "Adam; Eq. loss and its gradient by psfd_physics_loss (library FFTs, FP64 sums)"}


# ----------------------------------------------------------------------------- CPU oracle
class _Enough(Exception):
    pass


def oracle_layered_solve(prob, seed, pol, warm_iters, timed_iters, tol=TOL, maxit=400):
    """The FP64 oracle solving one mask at one polarisation the way the GPU path does (cold start,
    layered-background P, BiCGSTAB on A P y = b), timed: set-up (grid and TMM tables, fill, b, the
    per-mode blocks from 3 nz unit-source applies, their LU factors), then the iterations.  The
    solve runs until its residual history reaches tol and at least warm_iters + timed_iters
    iterations have run (maxit bounds it); the iteration time is the mean over the timed_iters
    iterations after the first warm_iters.  Returns (set-up s, s per iteration, iterations to tol)."""
    import torch
    from oracle import krylov as OK
    from oracle import psfd as O
    from paper_2607_25330_b300 import inputs as I
    a = I.mask_for(prob, seed)
    t0 = time.perf_counter()
    g = O.Grid(prob.to_dict(), prob.stack())
    fill = O.fill_fraction(a, prob.zprofile(), prob.sigma_px)
    b = O.source_b(g, fill, pol)
    mats = O.layered_blocks(g, fill)
    lu = torch.linalg.lu_factor(mats)
    del mats
    t_setup = time.perf_counter() - t0
    need = warm_iters + timed_iters
    stamps = []

    class History(list):
        def append(self, v):
            super().append(v)
            stamps.append(time.perf_counter())
            if (len(self) >= need and min(self) <= tol) or len(self) >= maxit:
                raise _Enough()

    h = History()
    try:
        OK.solve(lambda E: O.apply_A(g, E, fill), lambda X: O.apply_P_layered(g, fill, X, lu=lu), b,
                 tol=0.0, maxit=maxit, method="bicgstab", history=h)
    except _Enough:
        pass
    n_tol = next((i + 1 for i, v in enumerate(h) if v <= tol), None)
    if len(stamps) < 2:
        raise RuntimeError(f"oracle solve stopped after {len(stamps)} iterations")
    # the solve may stop early (a breakdown far below tol): time the iterations that ran
    last = min(need, len(stamps)) - 1
    first = min(max(warm_iters, 1), last) - 1
    t_iter = (stamps[last] - stamps[first]) / (last - first)
    return t_setup, t_iter, n_tol, len(h)


def cpu_baseline(args):
    import torch
    from paper_2607_25330_b300 import inputs as I
    prob = I.preset(args.workload)
    t_setup, t_iter, n_tol, ran = oracle_layered_solve(prob, args.warmup, prob.pols[0], 1, 3)
    if n_tol is None:
        return {"value": 0.0, "unit": "solves/s", "cores": torch.get_num_threads(), "kind": "oracle",
                "sample": f"FP64 oracle layered solve of one {args.workload} mask did not reach {TOL:g} in {ran} "
                          "iterations"}
    s = t_setup + n_tol * t_iter
    return {"value": 1.0 / s, "unit": "solves/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"one full FP64 oracle solve of one {args.workload} mask (TE, cold start, layered P, "
                      f"BiCGSTAB) to {TOL:g}: set-up incl. blocks and LU {t_setup:.1f} s, {n_tol} iterations "
                      f"to {TOL:g} (measured), {t_iter:.2f} s per iteration (mean of iterations 2-4); "
                      f"solves/s = 1 / (set-up + iterations x iteration time)",
            "seconds_per_solve": s, "iters_to_tol": n_tol}


def run_reference(args):
    """The oracle as the reference arm: one real FP64 solve of the bench's workload on the host
    cores; a step is one BiCGSTAB iteration (A P twice), timed after --warmup iterations."""
    import torch
    from paper_2607_25330_b300 import inputs as I
    prob = I.preset(args.workload)
    W = max(1, args.warmup)
    K = max(1, args.steps)
    t_setup, t_iter, n_tol, ran = oracle_layered_solve(prob, W, prob.pols[0], W, K, maxit=max(400, W + K))
    value = 1.0 / (t_setup + n_tol * t_iter) if n_tol else 0.0
    cb = {"value": value, "unit": "solves/s", "cores": torch.get_num_threads(), "kind": "oracle",
          "sample": f"one FP64 oracle solve of one {args.workload} mask (TE, cold start, layered P, BiCGSTAB): "
                    f"set-up incl. blocks and LU {t_setup:.1f} s; {n_tol} iterations to {TOL:g} (measured; the "
                    f"solve ran {ran}); a step = one iteration, {t_iter:.2f} s, timed over {K} iterations after "
                    f"{W}; solves/s = 1 / (set-up + iterations to tol x iteration time)"}
    return {"impl": "reference", "metric": "PSFD solves/s to rel. residual 1e-6 (warm start; cold alongside)",
            "value": value, "unit": "solves/s", "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * t_iter, "higher_is_better": True, "scaling": "weak",
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
    if args.profile_fno:
        print(json.dumps(run_profile_fno(args)), flush=True)
        return
    if args.train_step:
        print(json.dumps(run_train_step(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)

    def side_arm(key, fn):
        """Run one of the other workloads after the headline; a failure is recorded in its key (with
        the library's message) instead of losing the headline line."""
        import torch
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        try:
            out[key] = fn()
        except Exception as e:   # noqa: BLE001 -- reported in the JSON line
            out[key] = {"error": f"{type(e).__name__}: {e}"}
            print(f"bench: {key} failed: {e}", file=sys.stderr, flush=True)

    if rank == 0 and not args.skip_batch:
        side_arm("batch", lambda: run_batch(args))
    if rank == 0 and not args.skip_fine:
        side_arm("fine_grid", lambda: run_fine(args))
    if rank == 0 and not args.skip_train_step:
        # the differentiation workload: one physics-informed FNO training step (3 timed after 2)
        side_arm("train_step", lambda: run_train_step(args, steps=3, warmup=2))
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
