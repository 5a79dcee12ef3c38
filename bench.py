#!/usr/bin/env python
"""Benchmark of the boundary-integral hot path on one GPU (or N independent replicas).

Workload (default): the batched configuration -- 64 perturbed drops whose degrees p are drawn from
{16, 24, 32, 48} (PCG64 seed 3), radii U(0.8, 1.2), centres rejection-sampled in a 12^3 box with
nominal gaps >= 0.2, lambda ~ U(0.5, 10), R = 2, Q = 0.5, Ca_E = 0.1, Langmuir surfactant (beta 0.2,
x_s 0.5), uniform field E = z; inputs seeded and synthetic. One step is one midpoint time step of
Algorithm 1 (shbim_step, dt = 1e-3): two stages, each building the geometry and singular self rows of
all 64 drops, solving the electric system (Eq. galerkin_En), evaluating the charge potential and the
electric and interfacial forces (Eqs. el_force, interfacial_force, langmuir), solving the Stokes system
(Eq. main_eq) and forming the surfactant rate; GMRES stops at a relative residual of 1e-8 checked with
FP64-class sums (mixed precision by iterative refinement: FP32 compensated inner solves, double-float
residuals). Every operator application is one launch per kernel kind over all drops (tile lists over
drops of uneven degree), and every GMRES operator application a replayed CUDA graph.

Metric: target-source kernel pairs per second = operator applications in the step x
sum_i N_t(i) x sum_j N_s(j) / step time (self pairs counted as N_t N_s rotated pairs), and the time to a
1e-8 residual of the electric and Stokes solves, mixed precision against plain FP64 GMRES.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "target-source kernel pairs/s, GMRES time-to-1e-8 per step: mixed/batched vs FP64"
UNIT = "pairs/s"
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 rate (vector and tensor), 1/64 of the FP32 lane rate
# DRAM bytes (read + write) per launch of the pair kernel classes from one single-pass ncu capture of the
# same kernels on this workload (profiles/); None where the kernel has changed since its capture.
TRAFFIC = {"pairs_fp32": 11.9e6, "pairs_fp64class": None}
# the last capture of a class whose kernel has changed since (reported beside the null, not as traffic)
TRAFFIC_BEFORE_CHANGE = {"pairs_fp64class": {
    "bytes_per_launch": 46.3e6,
    "changed_since": "k_pairs_dq's powers of 1/r now come from the renormalised pair (arithmetic only, the "
                     "same loads); counters not taken again"}}
WORKLOAD_NAME = ("config 3: 64 drops, p in {16,24,32,48} (seed 3), radii U(0.8,1.2), 12^3 box, gaps >= 0.2, "
                 "lambda U(0.5,10), R=2, Q=0.5, Ca_E=0.1, Langmuir beta=0.2 x_s=0.5, E=z; one midpoint time "
                 "step (Algorithm 1) = 2 x (geometry + singular rows + electric solve + potential + forces + "
                 "Stokes solve + surfactant rate), GMRES to a 1e-8 residual checked in FP64-class arithmetic")


def batched_workload():
    return inputs.config3(seed=3)


def pairs_per_application(cfg) -> int:
    nt = sum((d.p + 1) * (2 * d.p + 2) for d in cfg.drops)
    ns = sum((2 * d.p + 2) * (4 * d.p + 4) for d in cfg.drops)
    return nt * ns


def cross_pairs(cfg) -> int:
    ns = sum((2 * d.p + 2) * (4 * d.p + 4) for d in cfg.drops)
    return sum((d.p + 1) * (2 * d.p + 2) * (ns - (2 * d.p + 2) * (4 * d.p + 4)) for d in cfg.drops)


def phys_of(S, cfg, Pe=math.inf):
    return S.phys(R=cfg.R, Q=cfg.Q, Ca_E=cfg.Ca_E, beta=0.2, x_s=0.5, E_u=tuple(cfg.E_u), E_q=cfg.E_quad,
                  inner_tol=1e-5, Pe=Pe)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- helpers

def cuda_time(torch, fn, stream=None):
    """(ms, result) of fn() between CUDA events on the current stream, synchronised on both sides."""
    stream = stream or torch.cuda.current_stream()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), r


def upload(torch, dev, cfg):
    x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=dev)
    g = torch.tensor(np.concatenate([d.gamma_coef for d in cfg.drops]), device=dev)
    return x, g


# FP64-class flops of the row build's weights stage per (target, rotated node) of a degree-p drop:
# Legendre sums of 9 fields (x, x_theta, x_phi/sin per component) 18 (p+1)(p+2)/2 FMAs per (target,
# rotated latitude), the four-fold Fourier synthesis 9 (N/4 + 1) 2p FMAs per (target, latitude),
# N = 2q + 2 rotated longitudes, and ~70 flops of pointwise geometry and kernel weights.
def weights_flops_per_unit(p: int) -> float:
    q = 2 * p + 1
    N = 2 * q + 2
    ntri = (p + 1) * (p + 2) // 2
    return 2 * (18 * ntri + 9 * (N // 4 + 1) * 2 * p) / N + 70


def roofline(cls_ms, cls_n, cls_work, cfg, peaks, dom=None):
    """Roofline of the dominant kernel class of one step (largest summed duration in the timing pass), or
    of class `dom`, from the method's own work: the all-pairs classes count the flops of the kernel
    formulas per target-source pair (shbim_kernel_work), the row build the FP64 flops of the weights
    stage."""
    if dom is None:
        dom = max(cls_ms, key=lambda k: cls_ms[k])
    ms, n = cls_ms[dom], cls_n[dom]
    ffma = peaks["ffma"]["value"]       # measured FP32 FMA rate, TFLOP/s
    out = {"kernel_class": dom, "launches": n, "avg_launch_ms": ms / max(1, n),
           "share_of_timed_kernel_time": ms / max(1e-9, sum(cls_ms.values())),
           "traffic": TRAFFIC.get(dom)}
    if dom in TRAFFIC_BEFORE_CHANGE:
        out["traffic_last_capture"] = TRAFFIC_BEFORE_CHANGE[dom]
    if dom in ("pairs_fp32", "pairs_fp64class"):
        ach = cls_work[dom] / (ms / 1e3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": ffma, "unit": "TFLOP/s", "frac": ach / ffma,
                    "peak_source": "FP32 FMA rate measured by this run's probe (shbim_probe_peak, 2 flops per FMA; "
                                   "MEASURED_PEAKS.json has no FP32 figure): of measured",
                    "work": "flops of the kernel formulas per target-source pair (Laplace SL 11, DL 19, Stokeslet 29, "
                            "stresslet 30, both 42) x pairs of different drops per launch",
                    "kernel": "k_pairs32 / k_pairs32_queue (FP32, compensated)" if dom == "pairs_fp32"
                              else "k_pairs_dq (double-float terms on quantised positions, FP32 pipe)"})
        if dom == "pairs_fp64class":
            out["frac_of_fp64_nominal"] = ach / FP64_NOMINAL_TFLOPS
        return out
    if dom == "self_weights":
        units = sum((d.p + 1) * (2 * d.p + 2) * (2 * d.p + 2) * (4 * d.p + 4) * weights_flops_per_unit(d.p)
                    for d in cfg.drops) * 2      # two geometries in the timing step
        ach = units / (ms / 1e3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": ffma, "unit": "TFLOP/s", "frac": ach / ffma,
                    "kernel": "k_self_weights_df (double-float on the FP32 pipe)",
                    "work": "FP64 flops of the weights stage per (target, rotated node) x units",
                    "peak_source": "measured FP32 FMA rate (the pipe the double-float arithmetic runs on)",
                    "frac_of_fp64_nominal": ach / FP64_NOMINAL_TFLOPS})
        return out
    out.update({"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                "note": "no algorithmic work model for this class"})
    return out


def class_names(S):
    return {S.K_SELF_WEIGHTS: "self_weights", S.K_SELF_ANALYSIS: "self_analysis", S.K_PAIRS: "pairs_fp32",
            S.K_SELF_GEMV: "self_gemv", S.K_SHT: "sht", S.K_SELF_ROTATION: "self_rotation",
            S.K_PAIRS_FP64CLASS: "pairs_fp64class", S.K_NEAR: "near"}


# --------------------------------------------------------------------------- own arm

def run_own(args):
    import torch
    import paper_1811_10270_gb300 as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    S.lib()
    if args.only:
        legs = {"pairs_at_scale": lambda: pairs_at_scale(S, torch, dev),
                "peaks": lambda: pipe_peaks(S),
                "learned": lambda: learned_warm_start(S, torch, dev, p=args.learned_p, n_train=args.learned_train,
                                                      n_test=args.learned_test, epochs=args.learned_epochs),
                "config2": lambda: config2_leg(S, torch, dev),
                "config3_fp64": lambda: time_to_solution_c3(S, torch, dev, fp64_full=True),
                "config5": lambda: config5_leg(S, torch, dev),
                "apps_config2": lambda: apps_config2(S, torch, dev),
                "apps_batched_p16": lambda: apps_batched_p16(S, torch, dev),
                "apps_batched": lambda: apps_batched(S, torch, dev)}
        print(json.dumps({args.only: legs[args.only]()}))
        return

    cfg = batched_workload()
    ps = [d.p for d in cfg.drops]
    lam = [d.lam for d in cfg.drops]
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8, gmres_restart=50)
    x, g = upload(torch, dev, cfg)
    nc = x.numel() // 3
    P = pairs_per_application(cfg)
    ph = phys_of(S, cfg)
    ctx.set_drops(ps, x, lam)
    x_out = torch.empty_like(x)
    g_out = torch.empty_like(g)
    dt = args.dt

    def step(xdev, gdev):
        a0 = ctx.operator_applications()
        err, its = ctx.step(ph, xdev, gdev, dt, x_out, g_out)
        return ctx.operator_applications() - a0, err, its

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step(x, g)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    apps_total = 0
    stats = []
    for _ in range(args.steps):
        r = step(x, g)
        apps_total += r[0]
        stats.append(r)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    if args.profile:
        ctx.close()
        print(json.dumps({"profile_run": True, "ms_per_step": ms / args.steps, "applications": apps_total,
                          "launches_before_timed": launches0, "launches_timed": launches}))
        return
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        a = torch.tensor([apps_total], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(a)
        apps_total = int(a.item())
    value = apps_total * P / (ms / 1e3)

    # Per-kernel-class durations and algorithmic work (phases, roofline): CUDA events around the kernel
    # classes on their launching streams, in one extra step with the second stream and the graphs off (in
    # the timed steps the row build's lanes overlap and GMRES applications replay graphs, which the
    # brackets do not see into).
    names = class_names(S)
    ctx.set_concurrency(False)
    ctx.set_graphs(False)
    ctx.set_timing(True)
    t_ms, _ = cuda_time(torch, lambda: step(x, g))
    cls_ms, cls_n, cls_work = {}, {}, {}
    for k, nm in names.items():
        cls_ms[nm], cls_n[nm] = ctx.kernel_stats(k)
        cls_work[nm] = ctx.kernel_work(k)
    ctx.set_timing(False)
    ctx.set_graphs(True)
    ctx.set_concurrency(not args.serial)

    # end to end through the public API: the state is copied in from pinned host memory every step and the
    # new state read back
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    x_pin = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops])).pin_memory()
    g_pin = torch.tensor(np.concatenate([d.gamma_coef for d in cfg.drops])).pin_memory()
    x_h = torch.empty(3 * nc, dtype=torch.float64).pin_memory()
    g_h = torch.empty(nc, dtype=torch.float64).pin_memory()

    def e2e_run():
        apps = 0
        for _ in range(e2e_steps):
            xd = x_pin.to(dev, non_blocking=True)
            gd = g_pin.to(dev, non_blocking=True)
            apps += step(xd, gd)[0]
            x_h.copy_(x_out, non_blocking=True)
            g_h.copy_(g_out, non_blocking=True)
        return apps

    ms_e2e, apps_e2e = cuda_time(torch, e2e_run)
    e2e_value = apps_e2e * P / (ms_e2e / 1e3)

    # reparametrisation after an accepted step (Section 2.2): 20 flow steps of the positions and the
    # concentration on the same layout, timed on its own (not part of the step above)
    xr, gr = x.clone(), g.clone()
    l0 = ctx.launch_count()
    ms_rep, e_rep = cuda_time(torch, lambda: ctx.reparametrize(xr, gr, steps=20, a=4.0, c=0.5))
    rep = {"flow_steps": 20, "a": 4.0, "c": 0.5, "ms": ms_rep, "ms_per_flow_step": ms_rep / 20,
           "launches": ctx.launch_count() - l0, "energy_ratio": e_rep[-1] / e_rep[0],
           "note": "shbim_reparametrize on the step's layout (positions and surfactant), FP64"}

    peaks = pipe_peaks(S)
    roof = roofline(cls_ms, cls_n, cls_work, cfg, peaks)
    roof_pairs = {k: roofline(cls_ms, cls_n, cls_work, cfg, peaks, dom=k) for k in ("pairs_fp32", "pairs_fp64class")}
    tts = time_to_solution_c3(S, torch, dev, fp64_full=args.fp64_full, ctx=ctx, cfg=cfg)
    apps_c3 = applications_by_kind(S, torch, dev, ctx, with_fp64=not args.no_fp64_apps)
    c2 = config2_leg(S, torch, dev) if not args.no_config2 else None
    learned = None if args.no_learned else learned_warm_start(S, torch, dev, p=args.learned_p, n_train=args.learned_train,
                                                              n_test=args.learned_test, epochs=args.learned_epochs)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+df32+f64",
        "data": "synthetic (seeded generators of the paper-shaped workloads)",
        "config": {"workload": WORKLOAD_NAME, "drops": len(ps),
                   "degrees": {str(p): ps.count(p) for p in sorted(set(ps))},
                   "targets": sum((p + 1) * (2 * p + 2) for p in ps),
                   "sources": sum((2 * p + 2) * (4 * p + 4) for p in ps),
                   "dt": args.dt, "precision": "mixed: FP32 compensated pair sums inside GMRES, double-float (FP64-class) "
                   "residuals and one-shot applications, FP64 Arnoldi",
                   "pairs_per_application": P,
                   "applications_per_step": apps_total / max(1, args.steps) / max(1, world),
                   "gmres_iters_per_step": stats[-1][2], "step_error_estimate": stats[-1][1],
                   "l2": "inputs larger than L2: the singular rows alone are ~10 GB, no flush needed",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "phase_ms_per_step": cls_ms,
        "timing_step_ms": t_ms,
        "kernel_timing": "phases and the roofline's launch durations: CUDA events around the kernel classes in one "
                         "extra step of the same workload with the library's second stream and CUDA graphs off",
        "time_to_1e-8": tts,
        "applications": apps_c3,
        "config2": c2,
        "learned_warm_start": learned,
        "reparametrization": rep,
        "roofline": roof,
        "roofline_pair_classes": roof_pairs,
        "pipe_peaks_measured": peaks,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": int(x_pin.numel() * 8 + g_pin.numel() * 8),
                "d2h_bytes_per_step": int(x_h.numel() * 8 + g_h.numel() * 8)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(gpu_config1_step(S, torch, dev))
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def applications_by_kind(S, torch, dev, ctx, with_fp64=True):
    """Metric 1 per kernel kind: one application of each layer operator (Laplace DL, SL, Stokes D, Stokes S)
    on the batched workload in FP32 (compensated), double-float and FP64, timed with CUDA events (second of
    two calls), as pairs/s with the algorithmic pair count."""
    nc, nt, ns = ctx.sizes()
    P = nt * ns
    rng = np.random.default_rng(1234)
    sig = torch.tensor(rng.standard_normal(nc), device=dev)
    f = torch.tensor(rng.standard_normal(3 * nc) / 4.0, device=dev)
    out = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    kinds = (("laplace_dl", lambda: ctx.eval_electric(S.LAPLACE_DL, sig, out[:nc])),
             ("laplace_sl", lambda: ctx.eval_electric(S.LAPLACE_SL, sig, out[:nc])),
             ("stokes_d", lambda: ctx.eval_stokes(None, f, out)),
             ("stokes_s", lambda: ctx.eval_stokes(f, None, out)))
    res = {"pairs_per_application": P}
    precs = [("fp32comp", S.FP32_COMP), ("df64", S.DF64)] + ([("fp64", S.FP64)] if with_fp64 else [])
    for pname, prec in precs:
        ctx.set_precision(prec)
        res[pname] = {}
        for kname, fn in kinds:
            fn()
            ms, _ = cuda_time(torch, fn)
            res[pname][kname] = {"ms": ms, "pairs_per_s": P / (ms / 1e3)}
    ctx.set_precision(S.FP32_COMP)
    res["pair_shapes_fp32"] = {k: list(ctx.pair_shape(i)[:2]) for i, k in enumerate(("dl", "sl", "sd", "s", "d"))}
    return res


def time_to_solution_c3(S, torch, dev, fp64_full=False, ctx=None, cfg=None):
    """Electric + Stokes solves to a relative residual of 1e-8 on one geometry of a many-drop workload:
    mixed precision (FP32 compensated inner GMRES, double-float residuals), plain GMRES with double-float
    sums, and plain GMRES with FP64 sums. The FP64 electric solve is timed in full; the FP64 Stokes solve
    is timed in full with fp64_full, otherwise as its set-up plus three Arnoldi steps (CUDA events) with
    the per-step time multiplied by the step count of the double-float solve (the same FP64-class
    arithmetic and convergence), labelled extrapolated."""
    own = ctx is None
    if own:
        cfg = batched_workload()
        ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8, gmres_restart=50)
        x, _ = upload(torch, dev, cfg)
        ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    nc, nt, ns = ctx.sizes()
    rhs_e = torch.empty(nc, device=dev, dtype=torch.float64)
    ctx.electric_rhs(cfg.E_u, rhs_e, E_q=cfg.E_quad)
    rng = np.random.default_rng(1234)
    f = torch.tensor(np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in cfg.drops]), device=dev)
    ctx.set_precision(S.DF64)
    rhs_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    ctx.eval_stokes(f, None, rhs_s)
    sol_e = torch.empty(nc, device=dev, dtype=torch.float64)
    sol_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    out = {"geometry": "one geometry of the workload", "rhs": "electric: R/(R+1) E.n; Stokes: S[f], f random "
           "smooth (N(0,1)/(n+1) per coefficient, seed 1234)"}
    ctx.set_precision(S.FP32_COMP)
    ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, sol_e, inner_tol=1e-5)     # graphs of this geometry
    ms_e, (ie, oe, re_) = cuda_time(torch, lambda: ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, sol_e, inner_tol=1e-5))
    ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, sol_s, inner_tol=1e-5)
    ms_s, (is_, os_, rs) = cuda_time(torch, lambda: ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, sol_s, inner_tol=1e-5))
    out["mixed"] = {"ms": ms_e + ms_s, "electric_ms": ms_e, "stokes_ms": ms_s, "inner_iters": [ie, is_],
                    "outer": [oe, os_], "resid_fp64class": [re_, rs]}
    ctx.set_precision(S.DF64)
    ms_de, (ide, rde) = cuda_time(torch, lambda: ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, sol_e))
    ms_ds, (ids, rds) = cuda_time(torch, lambda: ctx.gmres_solve(S.SYS_STOKES, rhs_s, sol_s))
    out["df64"] = {"ms": ms_de + ms_ds, "iters": [ide, ids], "resid": [rde, rds]}
    ctx.set_precision(S.FP64)
    ms_fe, (ife, rfe) = cuda_time(torch, lambda: ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, sol_e))
    if fp64_full:
        ms_fs, (ifs, rfs) = cuda_time(torch, lambda: ctx.gmres_solve(S.SYS_STOKES, rhs_s, sol_s))
        out["fp64"] = {"ms": ms_fe + ms_fs, "iters": [ife, ifs], "resid": [rfe, rfs], "stokes": "measured"}
    else:
        def begin_and_steps():
            ctx.gmres_begin(S.SYS_STOKES, rhs_s)
            for _ in range(3):
                ctx.gmres_step()
        ms_part, _ = cuda_time(torch, begin_and_steps)
        ms_one, _ = cuda_time(torch, lambda: ctx.gmres_step())
        ms_fs = ms_part + (ids - 3) * ms_one + ms_one      # + the final residual check of a solve
        out["fp64"] = {"ms": ms_fe + ms_fs, "iters": [ife, ids], "resid": [rfe, None],
                       "stokes": "extrapolated: set-up + 3 Arnoldi steps measured (%.0f ms), then %.0f ms per "
                                 "step x the double-float solve's %d steps" % (ms_part, ms_one, ids)}
    out["electric_fp64_ms"] = ms_fe
    out["stokes_fp64_ms"] = ms_fs
    ctx.set_precision(S.FP32_COMP)
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["speedup_df64_vs_fp64"] = out["fp64"]["ms"] / out["df64"]["ms"]
    if own:
        ctx.close()
    return out


def config2_leg(S, torch, dev, steps=5):
    """The two-drop workload (p = 32, 0.1 apart, lambda = 5): time step (mixed precision) and the time to a
    1e-8 residual of its electric + Stokes solves, mixed against plain FP64 (both measured in full)."""
    cfg = inputs.config2(p=32, seed=0, gap=0.1)
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
    x, g = upload(torch, dev, cfg)
    ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    ph = phys_of(S, cfg)
    xo, go = torch.empty_like(x), torch.empty_like(g)
    for _ in range(3):
        ctx.step(ph, x, g, 1e-3, xo, go)
    a0 = ctx.operator_applications()
    ms, _ = cuda_time(torch, lambda: [ctx.step(ph, x, g, 1e-3, xo, go) for _ in range(steps)])
    apps = (ctx.operator_applications() - a0) / steps
    P = pairs_per_application(cfg)
    nc = x.numel() // 3
    rhs_e = torch.empty(nc, device=dev, dtype=torch.float64)
    ctx.electric_rhs(cfg.E_u, rhs_e)
    rng = np.random.default_rng(1234)
    f = torch.tensor(np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in cfg.drops]), device=dev)
    ctx.set_precision(S.DF64)
    rhs_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    ctx.eval_stokes(f, None, rhs_s)
    sol_e, sol_s = torch.empty_like(rhs_e), torch.empty_like(rhs_s)
    res = {"workload": "two drops p=32 gap=0.1 seed 0 (config 2)", "ms_per_step": ms / steps,
           "pairs_per_s": apps * P / (ms / steps / 1e3), "applications_per_step": apps}
    for name, prec in (("mixed", S.FP32_COMP), ("df64", S.DF64), ("fp64", S.FP64)):
        ctx.set_precision(prec)

        def solve():
            if prec == S.FP32_COMP:
                return (ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, sol_e, inner_tol=1e-5),
                        ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, sol_s, inner_tol=1e-5))
            return ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, sol_e), ctx.gmres_solve(S.SYS_STOKES, rhs_s, sol_s)
        solve()
        t, r = cuda_time(torch, solve)
        res[name] = {"ms": t, "result": r}
    res["speedup_mixed_vs_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    ctx.close()
    return res


def apps_config2(S, torch, dev):
    """One application of each kernel kind (Laplace DL, SL, Stokes D, S) in FP32, double-float and FP64 on
    the two-drop workload (p = 32, gap 0.1): a short program of a few hundred launches, for profiling
    single kernels."""
    cfg = inputs.config2(p=32, seed=0, gap=0.1)
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
    x, _ = upload(torch, dev, cfg)
    ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    res = applications_by_kind(S, torch, dev, ctx, with_fp64=True)
    ctx.close()
    return res


def apps_batched_p16(S, torch, dev):
    """One application of each kernel kind (Laplace DL, SL, Stokes D, S) in FP32 and FP64-class arithmetic on
    64 drops of degree 16 in the batched workload's box (5.4e9 cross pairs, near correction off): a short
    program of a few hundred launches for profiling the all-pairs kernels at scale."""
    cfg = inputs.config3(seed=3, degrees=(16,))
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
    ctx.set_near(False)
    x, _ = upload(torch, dev, cfg)
    ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    res = applications_by_kind(S, torch, dev, ctx, with_fp64=False)
    ctx.close()
    return res


def apps_batched(S, torch, dev):
    """One application of each kernel kind in FP32 and FP64-class arithmetic on the batched workload itself
    (no FP64): a short program for capturing the pair kernels' DRAM traffic at full size."""
    cfg = batched_workload()
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
    x, _ = upload(torch, dev, cfg)
    ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    res = applications_by_kind(S, torch, dev, ctx, with_fp64=False)
    ctx.close()
    return res


def config5_leg(S, torch, dev):
    """16 drops of degree 64 in the quadrupole field (x, -y, 0), Pe = 10: geometry build, one mixed
    precision IMEX step (Algorithm 1) and the time to 1e-8, mixed vs FP64."""
    cfg = inputs.config5(seed=5)
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8, gmres_restart=50)
    x, g = upload(torch, dev, cfg)
    build_ms, _ = cuda_time(torch, lambda: ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops]))
    ph = phys_of(S, cfg, Pe=10.0)
    xo, go = torch.empty_like(x), torch.empty_like(g)
    a0 = ctx.operator_applications()
    ms, (err, its) = cuda_time(torch, lambda: ctx.step(ph, x, g, 1e-3, xo, go))
    res = {"workload": cfg.name, "geometry_build_ms": build_ms, "imex_step_pe10_ms": ms, "err_estimate": err,
           "gmres_iters": its, "operator_applications": ctx.operator_applications() - a0}
    res["time_to_1e-8"] = time_to_solution_c3(S, torch, dev, fp64_full=False, ctx=ctx, cfg=cfg)
    ctx.close()
    return res


# FP32 issue slots per pair of the FP32 kernels as implemented, counted from their source (hi/lo target
# offsets 6, r^2 3, kernel-specific terms, accumulation), the MUFU reciprocal square root extra; and the
# method's flops per pair (shbim_kernel_work)
PAIR_SLOTS = {"laplace_dl": 16, "laplace_sl": 10, "stokes_d": 23, "stokes_s": 21}
PAIR_FLOPS = {"laplace_dl": 19, "laplace_sl": 11, "stokes_d": 30, "stokes_s": 29}


def pairs_at_scale(S, torch, dev, reps: int = 10):
    """Throughput of the FP32 all-pairs kernels alone on 64 drops of degree 16 in a 12^3 box (5.5e9
    target-source pairs per application), each kernel kind timed by CUDA events around its launches, as
    pairs/s and as the method's flops per pair against the measured FP32 FMA rate."""
    cfg = inputs.config3(seed=3, degrees=(16,))
    ps = [d.p for d in cfg.drops]
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R)
    ctx.set_near(False)
    x, _ = upload(torch, dev, cfg)
    ctx.set_drops(ps, x, [d.lam for d in cfg.drops])
    nc, nt, ns = ctx.sizes()
    cross = cross_pairs(cfg)
    rng = np.random.default_rng(5)
    sig = torch.tensor(rng.standard_normal(nc), device=dev)
    f = torch.tensor(rng.standard_normal(3 * nc), device=dev)
    out = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    peak = pipe_peaks(S)["ffma"]["value"]
    res = {"workload": "64 drops p=16 (config-3 layout), cross pairs per application %d" % cross, "peak_tflops": peak}
    for name, fn in (("laplace_dl", lambda: ctx.eval_electric(S.LAPLACE_DL, sig, out[:nc])),
                     ("laplace_sl", lambda: ctx.eval_electric(S.LAPLACE_SL, sig, out[:nc])),
                     ("stokes_d", lambda: ctx.eval_stokes(None, f, out)),
                     ("stokes_s", lambda: ctx.eval_stokes(f, None, out))):
        fn()
        torch.cuda.synchronize()
        ctx.set_timing(True)
        for _ in range(reps):
            fn()
        ms, n = ctx.kernel_stats(S.K_PAIRS)
        ctx.set_timing(False)
        per = ms / max(1, n)
        ach = PAIR_FLOPS[name] * cross / (per / 1e3) / 1e12
        res[name] = {"pairs_per_s": cross / (per / 1e3), "ms_per_application": per, "method_tflops": ach,
                     "frac_of_measured_ffma": ach / peak, "issue_slots_per_pair": PAIR_SLOTS[name]}
    ctx.close()
    return res


def learned_warm_start(S, torch, dev, p: int = 32, n_train: int = 1000, n_test: int = 16, epochs: int = 60):
    """The learned warm start (config-4 style: two drops of degree p; the features, the network and its training
    run in the library's kernels). Trained on the method's own solutions of n_train seeds; on n_test held-out
    seeds the electric solve (field right-hand side) and the Stokes solve (right-hand side from the converged
    E_n, shbim_stokes_rhs) are timed to a 1e-8 residual checked in FP64-class arithmetic: mixed precision from
    zero, mixed precision from the network's guess (features and inference included), and plain FP64 GMRES
    from zero."""
    from paper_1811_10270_gb300 import warmstart
    t0 = time.perf_counter()
    X, Y, its0 = warmstart.generate(inputs.config2(p=p, seed=sd, gap=0.1) for sd in range(1, n_train + 1))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, hist = warmstart.train(X, Y, hidden=(512, 512, 512), epochs=epochs, batch=32, lr=1e-3)
    t_train = time.perf_counter() - t0
    kinds = ("zero", "learned", "fp64")
    ms = {sysn: {k: [] for k in kinds} for sysn in ("electric", "stokes")}
    its = {sysn: {k: [] for k in kinds} for sysn in ("electric", "stokes")}
    r0 = {"electric": [], "stokes": []}
    for sd in range(100000, 100000 + n_test):
        cfg = inputs.config2(p=p, seed=sd, gap=0.1)
        x, g = upload(torch, dev, cfg)
        nc = x.numel() // 3
        ph = warmstart.phys_of(cfg)
        ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
        ctx.set_drops([p, p], x, [d.lam for d in cfg.drops])
        rhs_e = torch.empty(nc, device=dev, dtype=torch.float64)
        ctx.electric_rhs(cfg.E_u, rhs_e)
        feat = torch.empty(ctx.warm_start_feature_count(), device=dev, dtype=torch.float32)
        En0 = torch.empty_like(rhs_e)
        u0 = torch.empty(3 * nc, device=dev, dtype=torch.float64)
        En = torch.empty_like(rhs_e)
        ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, En)          # graphs of this geometry; E_n for the Stokes rhs
        rhs_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
        ctx.stokes_rhs(ph, g, En, rhs_s)
        u = torch.empty_like(rhs_s)
        ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, u)
        for sysn, sysk, rhs, sol, guess in (("electric", S.SYS_ELECTRIC, rhs_e, En, En0),
                                           ("stokes", S.SYS_STOKES, rhs_s, u, u0)):
            for k in kinds:
                def run():
                    if k == "fp64":
                        ctx.set_precision(S.FP64)
                        it, _ = ctx.gmres_solve(sysk, rhs, sol)
                        ctx.set_precision(S.FP32_COMP)
                        return it
                    x0 = None
                    if k == "learned":
                        ctx.warm_start_features(x, g, ph, feat)
                        ctx.learned_guess(net, feat, rhs_e, En0, u0)
                        x0 = guess
                    inner, outer, _ = ctx.gmres_solve_refined(sysk, rhs, sol, x0=x0)
                    return inner
                t, it = cuda_time(torch, run)
                ms[sysn][k].append(t)
                its[sysn][k].append(it)
            r0[sysn].append(float(torch.linalg.norm(guess - sol) / torch.linalg.norm(sol)))
        ctx.close()
    net.close()
    return {"scale": "p=%d two-drop inputs (config-2 style), %d training solves, %d held out, %d epochs"
                     % (p, n_train, n_test, epochs),
            "generate_s": t_gen, "train_s": t_train, "final_loss_ratio": hist[-1] / hist[0],
            "mean_ms_to_1e-8": {s_: {k: float(np.mean(v)) for k, v in d.items()} for s_, d in ms.items()},
            "mean_iterations": {s_: {k: float(np.mean(v)) for k, v in d.items()} for s_, d in its.items()},
            "mean_guess_rel_error": {s_: float(np.mean(v)) for s_, v in r0.items()},
            "note": "zero and learned: mixed precision (FP32 inner GMRES, double-float residuals), iterations are "
                    "inner Arnoldi steps; fp64: plain FP64 GMRES from zero; learned includes features and inference"}


# outer iterations per probe: about 50 ms each on a GB300
PROBE_ITERS = {"ffma": 200000, "dfma": 3000, "rsqrt": 25000, "hmma_bf16": 300000, "dmma_f64": 3000}


def pipe_peaks(S):
    """Measured issue-bound rates of the pipes the kernels use (shbim_probe_peak)."""
    kinds = {"ffma": S.PROBE_FFMA, "dfma": S.PROBE_DFMA, "rsqrt": S.PROBE_RSQRT,
             "hmma_bf16": S.PROBE_HMMA_BF16, "dmma_f64": S.PROBE_DMMA_F64}
    out = {}
    for name, k in kinds.items():
        r, ms = S.probe_peak(k, PROBE_ITERS[name])
        out[name] = {"value": r / 1e12, "unit": "Tops/s" if name == "rsqrt" else "TFLOP/s", "ms": ms}
    return out


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample():
    """The FP64 oracle on a bounded sample of one application of the Laplace double layer on the batched
    workload, extrapolated to the whole application. The oracle's cost has two parts with different rates:
    the regular sums between drops (vectorised over sources) and the singular self rows, which it forms by
    direct evaluation on the rotated grid of each target. Sample: one drop of each degree; for each, its
    regular sums at 8 of its targets against the other sample drops' sources, and the self row of one of
    its targets. Returns (extrapolated application time, what was measured)."""
    from oracle import operators, quadrature, sh
    cfg = batched_workload()
    by_p = {}
    for j, d in enumerate(cfg.drops):
        by_p.setdefault(d.p, j)
    sample = [by_p[p] for p in sorted(by_p)]
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    geo = {j: operators.DropGeom(cfg.drops[j].xcoef, cfg.drops[j].p, cfg.drops[j].lam) for j in sample}
    t_geo = time.perf_counter() - t0
    sig = {j: inputs.random_density(cfg.drops[j].p, rng)[0] for j in sample}
    dens = {j: sh.sht_inverse(sig[j], geo[j].p, geo[j].q) for j in sample}
    reg_pairs, reg_s = 0, 0.0
    self_s = {}
    for i in sample:
        gi = geo[i]
        tsel = np.linspace(0, gi.nt - 1, 8).astype(int)
        t0 = time.perf_counter()
        for j in sample:
            if j == i:
                continue
            quadrature.regular_scalar("ladl", gi.x0[:, tsel], gi.n0[:, tsel], geo[j].xs, geo[j].ws, dens[j])
            reg_pairs += len(tsel) * geo[j].xs.shape[1]
        reg_s += time.perf_counter() - t0
        t0 = time.perf_counter()
        gi.rows("ladl", [int(tsel[3])])
        self_s[str(gi.p)] = time.perf_counter() - t0
    rate_reg = reg_pairs / reg_s
    # whole application: regular pairs at the measured rate, every target's self row at its degree's time
    cross = cross_pairs(cfg)
    t_self = sum((d.p + 1) * (2 * d.p + 2) * self_s[str(d.p)] for d in cfg.drops)
    t_app = cross / rate_reg + t_self
    return t_app, {"regular_pairs_per_s": rate_reg, "self_row_s_per_target": self_s, "sample_geometry_s": t_geo,
                   "sample_wall_s": t_geo + reg_s + sum(self_s.values())}


CONFIG1_PARAMS = dict(R=0.1, Q=1.0, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.0, 0.0, 1.0))


def oracle_config1_step():
    """One full time step of Algorithm 1 of the single unit-sphere drop (p = 16, Gamma = 1 + 0.1 Y_2^0,
    R = 0.1, Q = 1, E = z, dt = 1e-3) by the FP64 oracle, measured in full (wall seconds)."""
    from oracle import physics as P
    cfg = inputs.config1(16)
    d = cfg.drops[0]
    prm = P.Params(gmres_tol=1e-8, **CONFIG1_PARAMS)
    t0 = time.perf_counter()
    P.step([d.xcoef], [d.gamma_coef], [d.p], [d.lam], 1e-3, prm, near=False)
    return time.perf_counter() - t0


def gpu_config1_step(S, torch, dev, steps=5):
    """The same step on the GPU (FP64 context: one drop has no pair sums, every operator is its singular
    rows), milliseconds per step over `steps` steps after one warm-up step."""
    cfg = inputs.config1(16)
    ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-8)
    x, g = upload(torch, dev, cfg)
    ctx.set_drops([16], x, [1.0])
    ph = S.phys(inner_tol=1e-5, **CONFIG1_PARAMS)
    xo, go = torch.empty_like(x), torch.empty_like(g)
    ctx.step(ph, x, g, 1e-3, xo, go)
    ms, _ = cuda_time(torch, lambda: [ctx.step(ph, x, g, 1e-3, xo, go) for _ in range(steps)])
    ctx.close()
    return ms / steps


def cpu_baseline(gpu_c1_ms=None):
    """The oracle on its sample (oracle_sample) with all host cores available to its BLAS calls and with
    one thread, as pairs/s of one application of the batched workload (extrapolated); beside it the
    oracle's full time step of the single-drop workload, measured in full, against the GPU's."""
    cfg = batched_workload()
    P = pairs_per_application(cfg)
    t_all, info_all = oracle_sample()
    t_one, info_one = oracle_sample_one_thread()
    cores = threads_used()
    t_c1 = oracle_config1_step()
    c1 = {"workload": "single unit-sphere drop p=16, Gamma = 1 + 0.1 Y_2^0, R=0.1, Q=1, E=z, dt=1e-3 (config 1)",
          "oracle_step_s": t_c1, "gpu_step_ms": gpu_c1_ms,
          "gpu_speedup": (1e3 * t_c1 / gpu_c1_ms) if gpu_c1_ms else None,
          "note": "one full time step of Algorithm 1 measured in full on all host threads (the oracle is "
                  "elementwise numpy; one thread is within a few percent, see the sample above)"}
    return {"value": P / t_all, "unit": UNIT, "cores": cores, "kind": "oracle", "config1_step": c1,
            "sample": "FP64 numpy oracle, Laplace double layer of the batched workload: one drop per degree, "
                      "regular sums at 8 targets each against the other sample drops' sources and one target's "
                      "self row each; extrapolated to one whole application (%d pairs): %.0f s on %d threads, "
                      "%.0f s on 1 thread" % (P, t_all, cores, t_one),
            "extrapolated_application_s": {"all_cores": t_all, "one_core": t_one},
            "value_one_core": P / t_one, "measured": {"all_cores": info_all, "one_core": info_one}}


def oracle_sample_one_thread():
    """oracle_sample in a child interpreter whose BLAS pools are limited to one thread (the limit has to be
    set before numpy loads its BLAS)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = "import json, bench; t, info = bench.oracle_sample(); print(json.dumps([t, info]))"
    r = subprocess.run([sys.executable, "-c", code], cwd=os.path.dirname(os.path.abspath(__file__)), env=env,
                       capture_output=True, text=True, check=True)
    t, info = json.loads(r.stdout.strip().splitlines()[-1])
    return t, info


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(x.get("num_threads", 1)) for x in info)
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):   # untimed warm-up samples
        oracle_sample()
    vals = []
    P = pairs_per_application(batched_workload())
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t_app, info = oracle_sample()
        vals.append(P / t_app)
    wall = time.perf_counter() - t0
    v = float(np.mean(vals))
    cores = threads_used()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generators of the paper-shaped workloads)",
           "config": {"workload": WORKLOAD_NAME, "device": "host CPU cores (rank 0 only); no GPU work",
                      "step": "one bounded oracle sample of an application, extrapolated to the whole application"},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": UNIT,
                            "sample": "FP64 numpy oracle, Laplace double layer of the batched workload, one drop per "
                                      "degree (regular sums at 8 targets against the other sample drops, one self row "
                                      "each), extrapolated to one application"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config2", action="store_true", help="skip the two-drop leg")
    ap.add_argument("--no-fp64-apps", action="store_true", help="skip the FP64 single applications")
    ap.add_argument("--fp64-full", action="store_true", help="time the FP64 Stokes solve in full (minutes)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--learned-p", type=int, default=32, help="degree of the learned warm-start leg")
    ap.add_argument("--learned-train", type=int, default=1000, help="training solves of the learned leg")
    ap.add_argument("--learned-test", type=int, default=16, help="held-out solves of the learned leg")
    ap.add_argument("--learned-epochs", type=int, default=60, help="training epochs of the learned leg")
    ap.add_argument("--only", choices=["pairs_at_scale", "peaks", "learned", "config2", "config3_fp64", "config5",
                                       "apps_config2", "apps_batched_p16", "apps_batched"],
                    help="run one measurement leg alone and print its JSON")
    ap.add_argument("--serial", action="store_true",
                    help="operator applications on the caller's stream alone (no side-stream branches)")
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed steps (for launch lists under a profiler)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_own(args)


if __name__ == "__main__":
    main()
