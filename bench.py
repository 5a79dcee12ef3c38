#!/usr/bin/env python
"""Benchmark of the boundary-integral hot path on one GPU (or N independent replicas).

Workload (default): two perturbed unit drops of degree p = 32, centre gap 2.1 (surface gap
0.1), lambda = 5, R = 2, Q = 0.5, uniform field E = z (the two-drop configuration), inputs
seeded and synthetic. One step is one midpoint time step of Algorithm 1 (shbim_step), whose two stages each
build the geometry and singular self rows, solve the electric system (Eq. galerkin_En),
evaluate the charge potential, the electric and interfacial forces (Eqs. el_force,
interfacial_force, langmuir), solve the Stokes system (Eq. main_eq) and form the surfactant
rate; GMRES stops at an FP64 relative residual of 1e-8 (mixed precision by refinement).
Metric: target-source kernel pairs per second = operator applications in the step x
sum_i N_t(i) x sum_j N_s(j) / step time (self pairs counted as N_t N_s rotated pairs).

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
FP64_PEAK_TFLOPS = 1.25         # GB300 FP64 rate (vector and tensor), 1/64 of the FP32 lane rate
# DRAM bytes (read + write) per launch from one ncu capture of the same kernel and workload
# (profiles/row_build_kernels_two_drops_p32.md: launches of 1 100 and 1 078 targets, mean); to be
# dropped once the kernel changes after the capture.
TRAFFIC = {"self_weights_df": 1.175e9}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload(p: int = 32):
    cfg = inputs.config2(p=p, seed=0, gap=0.1)
    rng = np.random.default_rng(1234)
    f = [inputs.random_density(d.p, rng, 3) for d in cfg.drops]
    return cfg, f


def pairs_per_application(cfg) -> int:
    nt = sum((d.p + 1) * (2 * d.p + 2) for d in cfg.drops)
    q = [2 * d.p + 1 for d in cfg.drops]
    ns = sum((qq + 1) * (2 * qq + 2) for qq in q)
    return nt * ns


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
    if args.only == "pairs_at_scale":
        print(json.dumps({"pairs_at_scale": pairs_at_scale(S, torch, dev)}))
        return
    if args.only == "peaks":
        print(json.dumps({"pipe_peaks_measured": pipe_peaks(S)}))
        return
    if args.only == "learned":
        print(json.dumps({"learned_warm_start": learned_warm_start(S, torch, dev, p=args.learned_p,
                                                                   n_train=args.learned_train,
                                                                   n_test=args.learned_test)}))
        return
    if args.only in ("config3", "config5"):
        print(json.dumps({args.only: batched_leg(S, torch, dev, args.only)}))
        return

    cfg, f = workload(args.p)
    prec = S.FP32_COMP if args.precision == "fp32comp" else S.FP64
    ctx = S.Context(precision=prec, R=cfg.R, gmres_tol=1e-8, gmres_restart=50)
    ctx.set_concurrency(not args.serial)
    ps = [d.p for d in cfg.drops]
    lam = [d.lam for d in cfg.drops]
    x_host = np.concatenate([d.xcoef.ravel() for d in cfg.drops])
    g_host = np.concatenate([d.gamma_coef for d in cfg.drops])
    f_host = np.concatenate([a.ravel() for a in f])
    xc = torch.tensor(x_host, device=dev)
    gc = torch.tensor(g_host, device=dev)
    F = torch.tensor(f_host, device=dev)
    nc = sum((p + 1) ** 2 for p in ps)
    P = pairs_per_application(cfg)
    E = cfg.E_u
    ph = S.phys(R=cfg.R, Q=cfg.Q, Ca_E=cfg.Ca_E, beta=0.2, x_s=0.5, E_u=tuple(E), inner_tol=1e-5)
    ctx.set_drops(ps, xc, lam)
    x_out = torch.empty_like(xc)
    g_out = torch.empty_like(gc)
    rhs_e = torch.empty(nc, device=dev, dtype=torch.float64)
    rhs_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    En = torch.empty(nc, device=dev, dtype=torch.float64)
    u = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    dt = args.dt

    def step(xdev, gdev):
        a0 = ctx.operator_applications()
        err, its = ctx.step(ph, xdev, gdev, dt, x_out, g_out)
        return ctx.operator_applications() - a0, err, its

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step(xc, gc)
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
        r = step(xc, gc)
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
        print(json.dumps({"profile_run": True, "ms_per_step": ms / args.steps, "applications": sum(r[0] for r in stats)}))
        return
    # Per-kernel-class durations (phases, roofline) with CUDA events on the launching streams, in
    # the same number of extra steps with the library's second stream off: in the timed steps the
    # row build's two lanes overlap, so a kernel's bracketed time there includes the other lane's.
    ctx.set_concurrency(False)
    ctx.set_timing(True)
    for _ in range(args.steps):
        step(xc, gc)
    torch.cuda.synchronize()
    cls_ms = {}
    cls_n = {}
    names = {S.K_SELF_WEIGHTS: "self_weights", S.K_SELF_ANALYSIS: "self_analysis",
             S.K_PAIRS: "pairs", S.K_SELF_GEMV: "self_gemv", S.K_SHT: "sht",
             S.K_SELF_ROTATION: "self_rotation"}
    for k, nm in names.items():
        cls_ms[nm], cls_n[nm] = ctx.kernel_stats(k)
    ctx.set_timing(False)
    ctx.set_concurrency(not args.serial)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        a = torch.tensor([apps_total], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(a)
        apps_total = int(a.item())
    value = apps_total * P / (ms / 1e3)

    # end to end: the state is copied in from pinned host memory and the new state read back
    x_pin = torch.tensor(x_host).pin_memory()
    g_pin = torch.tensor(g_host).pin_memory()
    x_h = torch.empty(3 * nc, dtype=torch.float64).pin_memory()
    g_h = torch.empty(nc, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    apps_e2e = 0
    for _ in range(args.steps):
        xd = x_pin.to(dev, non_blocking=True)
        gd = g_pin.to(dev, non_blocking=True)
        r = step(xd, gd)
        apps_e2e += r[0]
        x_h.copy_(x_out, non_blocking=True)
        g_h.copy_(g_out, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    e2e_value = apps_e2e * P / (ms_e2e / 1e3)

    # the operator solves on the half-step geometry: right-hand sides for the comparison
    ctx.electric_rhs(E, rhs_e)
    ctx.eval_stokes(F, None, rhs_s, S.OUT_COEF)

    # time to a 1e-8 FP64 residual for both solves: mixed (refined) vs plain FP64 GMRES
    tts = time_to_solution(ctx, S, torch, stream, rhs_e, rhs_s, En, u)

    scale = pairs_at_scale(S, torch, dev) if not args.no_scale else None
    learned = learned_warm_start(S, torch, dev, p=args.learned_p, n_train=args.learned_train,
                                 n_test=args.learned_test) if not args.no_learned else None

    # roofline of the dominant kernel class (measured above with CUDA events)
    dom = max(cls_ms, key=lambda k: cls_ms[k])
    roof = roofline(dom, cls_ms[dom], cls_n[dom], cfg, args.steps, args.precision, P, apps_total)
    peaks = pipe_peaks(S)
    if roof.get("bound") == "alu" and "FP64" in roof.get("kernel", ""):
        roof["frac_of_measured_dfma"] = roof["achieved"] / peaks["dfma"]["value"]
    if roof.get("unit") == "Tinst/s":
        roof["frac_of_measured_ffma_issue"] = roof["achieved"] / (peaks["ffma"]["value"] / 2)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+df32+f64" if args.precision == "fp32comp" else "f64",
        "data": "synthetic",
        "config": {"workload": "two drops p=32 gap=0.1 (lambda=5, R=2, Q=0.5, Ca_E=0.1, Langmuir "
                               "beta=0.2 x_s=0.5, E=z): one midpoint time step (Algorithm 1) = 2 x "
                               "(geometry + singular rows + electric solve + potential + forces + "
                               "Stokes solve + surfactant rate), GMRES to an FP64 residual of 1e-8",
                   "dt": args.dt, "pair_sums": args.precision, "pairs_per_application": P,
                   "applications_per_step": apps_total / max(1, args.steps) / max(1, world),
                   "gmres_iters_per_step": stats[-1][2], "step_error_estimate": stats[-1][1],
                   "l2": "working set (singular rows 0.53 GB) exceeds the 129 MB L2; no flush",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "phase_ms_per_step": {k: v / args.steps for k, v in cls_ms.items()},
        "kernel_timing": "phases and the roofline's launch durations: CUDA events around the kernel classes in "
                         "%d extra steps of the same workload with the library's second stream off (in the timed "
                         "steps the row build's two lanes overlap); GMRES applications replayed from CUDA graphs "
                         "are not bracketed" % args.steps,
        "time_to_1e-8": tts,
        "pairs_at_scale": scale,
        "learned_warm_start": learned,
        "roofline": roof,
        "pipe_peaks_measured": peaks,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(x_host.nbytes + g_host.nbytes),
                "d2h_bytes_per_step": int(x_host.nbytes + g_host.nbytes)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.p, args.cpu_targets)
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


# FP32 pipe issue slots per pair of the all-pairs kernels, counted from their source (hi/lo
# offsets 6, r^2 3, kernel-specific terms, accumulation); the MUFU rsqrt is extra.
PAIR_SLOTS = {"laplace_dl": 16, "laplace_sl": 10, "stokes_sd": 29}


def pairs_at_scale(S, torch, dev, reps: int = 10):
    """Throughput of the FP32 all-pairs kernels on 64 drops of degree 16 in a 12^3 box (5.5e9
    target-source pairs per application): each kernel kind timed by CUDA events around its
    launches (classes of the library's kernel timing), as pairs/s and as a fraction of the
    FP32 pipe peak 152 SMs x 128 lanes x 2.07 GHz (2 flops per issue slot)."""
    cfg = inputs.config3(seed=3, degrees=(16,))
    ps = [d.p for d in cfg.drops]
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R)
    ctx.set_near(False)
    x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=dev)
    ctx.set_drops(ps, x, [d.lam for d in cfg.drops])
    nc, nt, ns = ctx.sizes()
    per_drop_t = [(p + 1) * (2 * p + 2) for p in ps]
    per_drop_s = [(2 * p + 2) * (4 * p + 4) for p in ps]
    cross = sum(a * (ns - b) for a, b in zip(per_drop_t, per_drop_s))
    rng = np.random.default_rng(5)
    sig = torch.tensor(rng.standard_normal(nc), device=dev)
    f = torch.tensor(rng.standard_normal(3 * nc), device=dev)
    out = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
    res = {"workload": "64 drops p=16 (config-3 layout), cross pairs per application %d" % cross}
    for name, fn in (("laplace_dl", lambda: ctx.eval_electric(S.LAPLACE_DL, sig, out[:nc])),
                     ("laplace_sl", lambda: ctx.eval_electric(S.LAPLACE_SL, sig, out[:nc])),
                     ("stokes_sd", lambda: ctx.eval_stokes(f, f, out))):
        fn()
        torch.cuda.synchronize()
        ctx.set_timing(True)
        for _ in range(reps):
            fn()
        ms, n = ctx.kernel_stats(S.K_PAIRS)
        ctx.set_timing(False)
        per = ms / max(1, n)
        ach = 2 * PAIR_SLOTS[name] * cross / (per / 1e3) / 1e12
        res[name] = {"pairs_per_s": cross / (per / 1e3), "ms_per_application": per,
                     "fp32_tflops_equiv": ach, "frac_of_fp32_peak": ach / peak}
    res["peak_tflops"] = peak
    ctx.close()
    return res


def learned_warm_start(S, torch, dev, p: int = 8, n_train: int = 600, n_test: int = 16):
    """The learned warm start (by default at reduced scale, p = 8 two-drop inputs; the network and its
    training run in the library's kernels): on held-out seeds, the electric solve to an FP64
    residual of 1e-8 from zero, from the sphere solution and from sphere + network --
    iterations, initial residual and time (CUDA events)."""
    from paper_1811_10270_gb300 import warmstart
    t0 = time.perf_counter()
    X, Y, _ = warmstart.generate(inputs.config2(p=p, seed=sd, gap=0.1) for sd in range(1, n_train + 1))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, hist = warmstart.train(X, Y, hidden=(512, 512, 512), epochs=150, batch=32, lr=1e-3)
    t_train = time.perf_counter() - t0
    names = ("zero", "sphere", "learned")
    it = {k: [] for k in names}
    r0 = {k: [] for k in names}
    ms = {k: 0.0 for k in names}
    stream = torch.cuda.current_stream()
    for sd in range(100000, 100000 + n_test):
        cfg = inputs.config2(p=p, seed=sd, gap=0.1)
        ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8)
        x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=dev)
        ctx.set_drops([p, p], x, [d.lam for d in cfg.drops])
        nc = x.numel() // 3
        rhs = torch.empty(nc, device=dev, dtype=torch.float64)
        ctx.electric_rhs(cfg.E_u, rhs)
        sol = torch.empty_like(rhs)
        ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs, sol)       # warm the graphs of this geometry
        for k in names:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            x0 = None
            if k == "sphere":
                x0 = 3.0 * (cfg.R + 1) / (cfg.R + 2) * rhs
            elif k == "learned":
                x0 = torch.empty_like(rhs)
                S.electric_warm_start(ctx, net, x, rhs, x0)
            inner, outer, res = ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs, sol, x0=x0)
            b.record(stream)
            torch.cuda.synchronize()
            ms[k] += a.elapsed_time(b)
            it[k].append(inner)
            if x0 is None:
                r0[k].append(1.0)
            else:
                Lx = torch.empty_like(rhs)
                ctx.eval_electric(S.LAPLACE_DL, x0, Lx, S.OUT_COEF)
                r = rhs - (0.5 * x0 - (cfg.R - 1) / (cfg.R + 1) * Lx)
                r0[k].append(float(torch.linalg.norm(r) / torch.linalg.norm(rhs)))
        ctx.close()
    net.close()
    return {"scale": "p=%d two-drop inputs, %d training solves, %d held out%s" % (
                p, n_train, n_test, "" if (p == 32 and n_train >= 20000) else " (reduced from 20 000 solves at p = 32)"),
            "train_s": t_train, "generate_s": t_gen, "final_loss_ratio": hist[-1] / hist[0],
            "mean_inner_iters": {k: float(np.mean(v)) for k, v in it.items()},
            "mean_initial_resid": {k: float(np.mean(v)) for k, v in r0.items()},
            "mean_ms_to_1e-8": {k: v / n_test for k, v in ms.items()}}


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


def batched_leg(S, torch, dev, name):
    """The many-drop workloads on one GPU, each measured once with CUDA events:
    config3 = 64 drops of degree 16/24/32/48 (uniform field), config5 = 16 drops of degree 64 in
    the quadrupole field (x, -y, 0). Reports the geometry build (shapes, singular rows, near
    pairs), one application of each layer operator in FP32 (compensated) and FP64 with the
    algorithmic pair count sum_i N_t(i) * sum_j N_s(j), and the electric and Stokes solves to an
    FP64 residual of 1e-8 from zero, mixed precision vs plain FP64; config5 also times one
    mixed-precision IMEX step at Pe = 10 (Algorithm 1)."""
    cfg = inputs.config3(seed=3) if name == "config3" else inputs.config5(seed=5)
    ps = [d.p for d in cfg.drops]
    lam = [d.lam for d in cfg.drops]
    stream = torch.cuda.current_stream()

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = None
        for _ in range(reps):
            r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, r

    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-8, gmres_restart=50)
    x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=dev)
    g = torch.tensor(np.concatenate([d.gamma_coef for d in cfg.drops]), device=dev)
    build_ms, _ = timed(lambda: ctx.set_drops(ps, x, lam))
    nc, nt, ns = ctx.sizes()
    pairs = nt * ns
    rng = np.random.default_rng(1234)
    sig = torch.tensor(rng.standard_normal(nc), device=dev)
    f = torch.tensor(rng.standard_normal(3 * nc) / 4.0, device=dev)
    out = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    res = {"workload": cfg.name, "drops": len(ps), "degrees": sorted(set(ps)), "ncoef": nc,
           "targets": nt, "sources": ns, "pairs_per_application": pairs, "near_pairs": ctx.near_pairs(),
           "geometry_build_ms": build_ms}
    kinds = (("laplace_dl", lambda: ctx.eval_electric(S.LAPLACE_DL, sig, out[:nc])),
             ("laplace_sl", lambda: ctx.eval_electric(S.LAPLACE_SL, sig, out[:nc])),
             ("stokes_sd", lambda: ctx.eval_stokes(f, f, out)))
    for pname, prec, reps in (("fp32comp", S.FP32_COMP, 3), ("df64", S.DF64, 1), ("fp64", S.FP64, 1)):
        ctx.set_precision(prec)
        res[pname] = {}
        for kname, fn in kinds:
            fn()                                    # first launch of a kind tunes its shape
            ms, _ = timed(fn, reps)
            res[pname][kname] = {"ms_per_application": ms, "pairs_per_s": pairs / (ms / 1e3)}
    res["pair_shapes"] = [ctx.pair_shape(k)[:2] for k in range(3)]
    # right-hand sides: the field term of the electric system; S[f] for Stokes
    rhs_e = torch.empty(nc, device=dev, dtype=torch.float64)
    ctx.electric_rhs(cfg.E_u, rhs_e, E_q=cfg.E_quad)
    ctx.set_precision(S.DF64)
    rhs_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    ctx.eval_stokes(f, None, rhs_s)
    sol_e = torch.empty(nc, device=dev, dtype=torch.float64)
    sol_s = torch.empty(3 * nc, device=dev, dtype=torch.float64)
    tts = {}
    ctx.set_precision(S.FP32_COMP)
    ms, (ie, oe, re_) = timed(lambda: ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, sol_e, inner_tol=1e-5))
    tts["electric_mixed"] = {"ms": ms, "inner_iters": ie, "outer": oe, "resid": re_}
    ms, (is_, os_, rs) = timed(lambda: ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, sol_s, inner_tol=1e-5))
    tts["stokes_mixed"] = {"ms": ms, "inner_iters": is_, "outer": os_, "resid": rs}
    ctx.set_precision(S.FP64)
    ms, (ie, re_) = timed(lambda: ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, sol_e))
    tts["electric_fp64"] = {"ms": ms, "iters": ie, "resid": re_}
    ms, (is_, rs) = timed(lambda: ctx.gmres_solve(S.SYS_STOKES, rhs_s, sol_s))
    tts["stokes_fp64"] = {"ms": ms, "iters": is_, "resid": rs}
    ctx.set_precision(S.DF64)
    ms, (ie, re_) = timed(lambda: ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, sol_e))
    tts["electric_df64"] = {"ms": ms, "iters": ie, "resid": re_}
    ms, (is_, rs) = timed(lambda: ctx.gmres_solve(S.SYS_STOKES, rhs_s, sol_s))
    tts["stokes_df64"] = {"ms": ms, "iters": is_, "resid": rs}
    tts["speedup_mixed_vs_fp64"] = ((tts["electric_fp64"]["ms"] + tts["stokes_fp64"]["ms"])
                                    / (tts["electric_mixed"]["ms"] + tts["stokes_mixed"]["ms"]))
    res["time_to_1e-8"] = tts
    if name == "config5":
        ctx.set_precision(S.FP32_COMP)
        ph = S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=tuple(cfg.E_u), E_q=cfg.E_quad,
                    inner_tol=1e-5, Pe=10.0)
        xo, go = torch.empty_like(x), torch.empty_like(g)
        a0 = ctx.operator_applications()
        ms, (err, its) = timed(lambda: ctx.step(ph, x, g, 1e-3, xo, go))
        res["imex_step_pe10"] = {"ms": ms, "dt": 1e-3, "err_estimate": err, "gmres_iters": its,
                                 "operator_applications": ctx.operator_applications() - a0}
    ctx.close()
    return res


def time_to_solution(ctx, S, torch, stream, rhs_e, rhs_s, En, u, reps=3):
    """Electric + Stokes solves to a relative residual of 1e-8 on the current geometry: plain
    GMRES with native FP64 sums, plain GMRES with double-float sums (FP64-class accuracy on the
    FP32 pipe), and mixed precision (FP32 compensated inner GMRES, double-float refinement)."""
    out = {}
    for name in ("fp64", "df64", "mixed"):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if name in ("fp64", "df64"):
                ctx.set_precision(S.FP64 if name == "fp64" else S.DF64)
                ie, re_ = ctx.gmres_solve(S.SYS_ELECTRIC, rhs_e, En)
                is_, rs = ctx.gmres_solve(S.SYS_STOKES, rhs_s, u)
                info = {"iters": [ie, is_], "resid": [re_, rs]}
            else:
                ctx.set_precision(S.FP32_COMP)
                ie, oe, re_ = ctx.gmres_solve_refined(S.SYS_ELECTRIC, rhs_e, En, inner_tol=1e-5)
                is_, os_, rs = ctx.gmres_solve_refined(S.SYS_STOKES, rhs_s, u, inner_tol=1e-5)
                info = {"inner_iters": [ie, is_], "outer": [oe, os_], "resid": [re_, rs]}
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            if best is None or ms < best[0]:
                best = (ms, info)
        out[name] = {"ms": best[0], **best[1]}
    ctx.set_precision(S.FP32_COMP)
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["speedup_df64_vs_fp64"] = out["fp64"]["ms"] / out["df64"]["ms"]
    return out


# FP32 instruction slots of the double-float operations of csrc/dfloat.cuh, counted from the source:
# multiply-accumulate into a running sum 12, product 7, sum / difference 11, 3-term dot product 31,
# reciprocal square root 28 (one MUFU seed + Newton step), square 7.
DF_MAC, DF_MUL, DF_ADD, DF_DOT3, DF_RSQRT, DF_SQR = 12, 7, 11, 31, 28, 7
# per rotated node: tangents' cross product, J and n, offset and 1/r, the 14 weights
DF_WEIGHTS_PER_NODE = (6 * DF_MUL + 3 * DF_ADD + DF_DOT3 + DF_RSQRT + DF_MUL + 3 * DF_MUL + 3 * DF_ADD
                       + DF_DOT3 + DF_RSQRT + DF_SQR + 3 * DF_MUL + DF_DOT3 + 6 + 3 * DF_MUL + 2 * DF_MUL
                       + DF_DOT3 + 2 * DF_MUL + 3 * DF_MUL + 6 * DF_MUL + 3 * DF_ADD + 3 * DF_MUL + 6 * DF_MUL)
FP32_ISSUE_TINST = SM_COUNT * FP32_LANES_PER_SM * 2.07e9 / 1e12   # FP32 lane instructions / s


def roofline(dom, ms, n, cfg, steps, precision, P, apps, rows_df=True):
    p = cfg.drops[0].p
    q = 2 * p + 1
    nt = (p + 1) * (2 * p + 2)
    ns = (q + 1) * (2 * q + 2)
    N = 2 * q + 2
    Q4 = N // 4
    ntri = (p + 1) * (p + 2) // 2
    # FP64 flops per (target, rotated node) of the weights stage: Legendre sums 18 (p+1)(p+2)/2
    # FMA per (target, latitude); four-fold Fourier synthesis 9 (N/4+1) 2p FMA per (target,
    # latitude); ~70 flops of pointwise geometry and kernel weights. FMA = 2 flops.
    fp64_per_unit = 2 * (18 * ntri + 9 * (Q4 + 1) * 2 * p) / N + 70
    units_w = sum(nt * ns for _ in cfg.drops) * steps * 2   # two geometries per step
    if dom == "self_weights" and rows_df:
        per_unit = (18 * ntri * DF_MAC + 9 * (Q4 + 1) * (2 * p * DF_MAC + 4 * 3 + 4 * DF_ADD
                                                            + 4 * (DF_MUL + 2 * DF_ADD))) / N \
            + DF_WEIGHTS_PER_NODE
        ach = per_unit * units_w / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "k_self_weights_df (double-float on the FP32 pipe)",
                "achieved": ach, "peak": FP32_ISSUE_TINST, "unit": "Tinst/s", "frac": ach / FP32_ISSUE_TINST,
                "traffic": TRAFFIC.get("self_weights_df"), "launches": n, "avg_launch_ms": ms / max(1, n),
                "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (derived; measured FFMA issue in "
                               "pipe_peaks_measured)",
                "per_unit_fp32_instructions": per_unit, "unit_of_work": "(target, rotated source node)",
                "fp64_equivalent_tflops": fp64_per_unit * units_w / (ms / 1e3) / 1e12,
                "fp64_equivalent_note": "the FP64 build's flops at this kernel's speed; FP64 peak 1.25"}
    if dom == "self_weights":
        ach = fp64_per_unit * units_w / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "k_self_weights (FP64)", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": TRAFFIC.get("self_weights"), "launches": n, "avg_launch_ms": ms / max(1, n),
                "peak_source": "GB300 FP64 rate 1.25 TFLOP/s (nominal)",
                "per_unit_flops": fp64_per_unit, "unit_of_work": "(target, rotated source node)"}
    units_a = sum(nt * ns * 14 for _ in cfg.drops) * steps * 2
    if dom == "self_analysis" and rows_df:
        # per (target, component, node): folds 4 adds per Q4 nodes, 2(p+1)(Q4-1) MACs per row of N
        # nodes, Legendre 2 ntri (q+1) MACs per item over Ns nodes
        per_unit = (4 * Q4 * DF_ADD + 2 * (p + 1) * (Q4 - 1) * DF_MAC) / N + 2 * ntri * (q + 1) * DF_MAC / ns
        ach = per_unit * units_a / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "k_analysis_f4_df/leg_df (double-float on the FP32 pipe)",
                "achieved": ach, "peak": FP32_ISSUE_TINST, "unit": "Tinst/s", "frac": ach / FP32_ISSUE_TINST,
                "traffic": None, "launches": n, "avg_launch_ms": ms / max(1, n),
                "per_unit_fp32_instructions": per_unit, "unit_of_work": "(target, component, rotated node)"}
    if dom == "self_analysis":
        per_unit = (2 * (2 * (p + 1) * (Q4 - 1)) + N + 2 * 2 * ntri) / N
        ach = per_unit * units_a / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "k_analysis_fourier4/legendre (FP64)", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": None, "launches": n, "avg_launch_ms": ms / max(1, n),
                "per_unit_flops": per_unit, "unit_of_work": "(target, component, rotated node)"}
    if dom == "pairs":
        per_pair = 20
        pk = SM_COUNT * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
        cross = P - sum(((d.p + 1) * (2 * d.p + 2)) * ((2 * d.p + 2) * (4 * d.p + 4)) for d in cfg.drops)
        ach = per_pair * cross * apps / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "k_pairs (FP32)", "achieved": ach, "peak": pk,
                "unit": "TFLOP/s", "frac": ach / pk, "traffic": None, "launches": n,
                "avg_launch_ms": ms / max(1, n)}
    return {"bound": "hbm", "kernel": dom, "achieved": None, "peak": None, "unit": "GB/s",
            "frac": None, "traffic": None, "launches": n, "avg_launch_ms": ms / max(1, n)}


# --------------------------------------------------------------------------- CPU oracle

def cpu_baseline(p: int, targets_per_drop: int):
    """The FP64 oracle timed on a bounded sample of the same workload: the electric double
    layer (self rows + regular sums from the other drop) at a few targets per drop."""
    from oracle import operators
    cfg, _ = workload(p)
    rng = np.random.default_rng(7)
    sig = [inputs.random_density(d.p, rng)[0] for d in cfg.drops]
    t0 = time.perf_counter()
    sysm = operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in cfg.drops])
    ns_tot = sum(d.xs.shape[1] for d in sysm.drops)
    done = 0
    for i, d in enumerate(sysm.drops):
        sel = np.linspace(0, d.nt - 1, targets_per_drop).astype(int)
        sysm.laplace_targets("ladl", sig, i, sel)
        done += len(sel) * ns_tot
    dt = time.perf_counter() - t0
    cores = threads_used()
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "electric double layer at %d targets per drop of the p=%d two-drop "
                      "workload (geometry set-up included), %.1f s" % (targets_per_drop, p, dt)}


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
    vals = []
    for _ in range(args.warmup):   # untimed warm-up samples (2 targets per drop each)
        cpu_baseline(args.p, 2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.p, args.cpu_targets))
    wall = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "two drops p=%d gap=0.1, FP64 CPU oracle on a bounded sample" % args.p,
                      "device": "host CPU cores (rank 0 only); no GPU work"},
           "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": vals[-1]["sample"],
                            "value": v, "unit": UNIT},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--precision", default="fp32comp", choices=["fp32comp", "fp64"])
    ap.add_argument("--p", type=int, default=32)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--cpu-targets", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scale", action="store_true", help="skip the 64-drop all-pairs measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--learned-p", type=int, default=8, help="degree of the learned warm-start leg")
    ap.add_argument("--learned-train", type=int, default=600, help="training solves of the learned leg")
    ap.add_argument("--learned-test", type=int, default=16, help="held-out solves of the learned leg")
    ap.add_argument("--only", choices=["pairs_at_scale", "config3", "config5", "peaks", "learned"],
                    help="run one measurement leg alone and print its JSON (for profiling)")
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
