"""Benchmark of the hot path: iterations of Algorithm 8 (one-step FB, ramp
preconditioner of Sec. 3.1) on the large single-solve workload (N = 384^3,
180 angles, T = 1.5, FP32-Kahan wavefields, FP64 reductions).

One step = one FB iteration = W (1344 leapfrog steps) + P + residual + Lambda
+ P^T + W^T (1344 steps) + the fused prox update with FP64 norms.  The metric
is voxel-steps per second (2 Nt N^3 per iteration over the device time), with
FB iterations per second alongside.  Prints ONE JSON line; unless
--no-extras, the line also carries the FP32-vs-FP64 comparison on the 128^3
solve, the measured FMA rates of the FP64 and FP32 pipes, a short serving-mix
run (p50 / p99, recons/s) and served FP32 against plain FP64 reconstructions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cfg5|cfg2|cfg1] [--precision fp32-kahan|fp32|fp64]
  python bench.py --mode op --op wave --n 384 --op-steps 12 --path 3   # one operation

Multi-GPU: the reconstruction does not shard across GPUs; N GPUs run N
independent replicas (one reconstruction each) and `value` is the sum.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant leapfrog kernel, taken from one ncu capture of that kernel on
# the same grid, keyed by (workload, precision, kernel).  An entry is dropped
# whenever its kernel changes, until it has been captured again.
NCU_TRAFFIC = {("cfg2", "fp32-kahan", "resident"): 17.151232e6,
               ("cfg5", "fp32-kahan", "two-step"): 1541.066496e6,
               ("cfg5", "fp32", "two-step"): 1095.204864e6}

# algorithmic FP32 operations per point-step of the difference-form update:
# 12 subtractions, 10 additions and one FMA (2) for 12 h^2 L4 p, then the
# Kahan increment (FMA + 4 adds) or the three-term update (FMA + 2 adds)
FLOP_PER_POINT_STEP = {"fp32-kahan": 30, "fp32": 28}
# FP64 pipe instructions per point-step of the FP64 leapfrog: 10 additions
# and 2 FMAs for 12 h^2 L4 p, two FMAs for the three-term update
FP64_OPS_PER_POINT_STEP = 14
# FP32 CUDA-core lanes: 152 SMs x 128
FP32_LANES = 152 * 128

WORKLOADS = {
    "cfg5": dict(cfg=5, label="large single solve N=384^3, 180 angles, T=1.5, 200 balls + 5 "
                              "tubes, GRF sound speed, ramp-preconditioned FB"),
    "cfg2": dict(cfg=2, label="single solve N=128^3, 90 angles, T=1.2, 20 balls, GRF sound speed"),
    "cfg1": dict(cfg=1, label="small solve N=32^3, 24 angles, T=1"),
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"ffpat_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, units_per_step, dev_ms_local, device=None):
    """Whole-job throughput of `world` independent replicas that each ran
    `steps` steps of `units_per_step` units: all ranks' units over the slowest
    rank's time.  Returns (value per second, slowest time in ms)."""
    slowest = max_over_ranks(dev_ms_local, world, device)
    return world * steps * units_per_step / (slowest / 1e3), slowest


def make_problem(args):
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import config
    wl = WORKLOADS[args.workload]
    w = config(wl["cfg"])
    prec = {"fp32-kahan": F.FP32_KAHAN, "fp32": F.FP32, "fp64": F.FP64}[args.precision]
    prob = F.problem(w.n, w.T, w.n_angles, prec, w.precond)
    return w, wl, prob


def workload_config(w, wl, nt, precision, world):
    """The `config` object of both arms' lines: the workload by name and sizes."""
    return {"workload": wl["label"], "n": w.n, "n_angles": w.n_angles, "T": w.T, "nt": nt,
            "precision": precision, "precond": "ramp" if w.precond else "identity",
            "fb_iteration": "W + P + residual + Lambda + P^T + W^T + prox update",
            "l2": "inputs larger than L2 and flushed (256 MB write) between timed steps",
            "parallelism": "replicas" if world > 1 else "single"}


def oracle_sample(w, seconds_target=10.0):
    """Time the oracle's wave operator (the dominant loop) on the workload's
    grid for a bounded number of leapfrog steps; returns voxel-steps/s."""
    import numpy as np
    import oracle.oracle as o
    nt, dt = o.time_steps(w.n, w.T, w.cfl, float(w.c.max()))
    kap = o.kappa(w.n, dt, w.c)
    t0 = time.perf_counter()
    o.wave(kap, w.h, 2)
    probe = time.perf_counter() - t0
    steps = int(max(2, min(nt, seconds_target / max(probe / 2, 1e-6))))
    t0 = time.perf_counter()
    out = o.wave(kap, w.h, steps)
    el = time.perf_counter() - t0
    assert np.isfinite(out).all()
    return steps * float(w.n) ** 3 / el, steps, el, o.num_threads()


def run_reference(args):
    world, rank, local = dist_init(args)
    if rank != 0:
        return 0
    import oracle.oracle as o
    o.build()
    w, wl, prob = make_problem(args)
    # each step is a bounded sample: the whole run stays within a few minutes
    # whatever --steps is (about 150 s of timed oracle work at most)
    per_step = min(args.ref_seconds, max(0.5, 150.0 / max(args.steps, 1)))
    for _ in range(args.warmup):
        oracle_sample(w, seconds_target=min(1.0, per_step))
    vals, total_vs, total_s = [], 0.0, 0.0
    for _ in range(args.steps):
        v, steps, el, cores = oracle_sample(w, seconds_target=per_step)
        total_vs += steps * float(w.n) ** 3
        total_s += el
    value = total_vs / total_s
    line = {
        "impl": "reference", "metric": "voxel-steps/s", "value": value, "unit": "voxel-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, wl, o.time_steps(w.n, w.T, w.cfl, float(w.c.max()))[0],
                                  "f64 (the oracle)", 1),
        "cpu_baseline": {"value": value, "unit": "voxel-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 CPU oracle wave operator W, {steps} leapfrog steps on "
                                   f"the {w.n}^3 grid per step (the FB iteration's dominant loop)"},
        "e2e": {"value": value, "unit": "voxel-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build_lib.build()
    F.lib()
    w, wl, prob = make_problem(args)
    dt = F.torch_dtype(prob)
    c = torch.as_tensor(w.c, device=dev).to(dt)
    h_true = torch.as_tensor(w.h, device=dev).to(dt)
    # synthetic data g = A h + noise, computed by the library in FP64
    p64 = F.problem(w.n, w.T, w.n_angles, F.FP64, w.precond)
    g64 = F.forward(p64, torch.as_tensor(w.c, device=dev), torch.as_tensor(w.h, device=dev))
    g = torch.as_tensor(add_noise(g64.cpu().numpy(), w.noise, w.noise_rel), device=dev).to(dt)
    del g64
    ws = F.workspace(prob, dev)
    nt, dtime, _ = F.problem_info(prob, float(w.c.astype(np.float32).max()
                                              if prob.precision != F.FP64 else w.c.max()))
    v0 = torch.ones_like(h_true)
    L = F.opnorm(prob, c, v0, iters=20, ws=ws)
    step = 1.0 / L
    h = torch.zeros_like(h_true)
    # inputs larger than L2 at 384^3; the 256 MB write flushes L2 between
    # timed steps at every size
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        F.fb_solve(prob, c, g, w.lam, step, 1, h=h, ws=ws, history=False)
    torch.cuda.synchronize()

    # ---- timed region: exactly K FB iterations, L2 flushed between them
    F.profile_enable(True)
    F.profile_read()
    launches0 = F.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("ffpat_timed")
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            F.fb_solve(prob, c, g, w.lam, step, 1, h=h, ws=ws, history=False)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        torch.cuda.nvtx.range_pop()
    barrier(world)
    prof = F.profile_read()
    launches = F.launch_count() - launches0
    F.profile_enable(False)
    vs_per_iter = 2.0 * nt * float(w.n) ** 3
    value, dev_ms = replica_throughput(world, args.steps, vs_per_iter,
                                       sum(a.elapsed_time(b) for a, b in ev), dev)
    clocks = clk.summary()

    # ---- end to end through the public API with host buffers
    c_h = torch.as_tensor(w.c).to(dt).pin_memory()
    g_h = g.cpu().pin_memory()
    h_h = torch.zeros_like(h_true, device="cpu").pin_memory()
    out_h = torch.empty_like(h_h).pin_memory()
    c_d, g_d, h_d = torch.empty_like(c), torch.empty_like(g), torch.empty_like(h)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c_d.copy_(c_h, non_blocking=True)
        g_d.copy_(g_h, non_blocking=True)
        h_d.copy_(h_h, non_blocking=True)
        F.fb_solve(prob, c_d, g_d, w.lam, step, 1, h=h_d, ws=ws, history=False)
        out_h.copy_(h_d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    esz = 8 if prob.precision == F.FP64 else 4
    h2d = (2 * w.n**3 + w.n_angles * w.n**2) * esz
    d2h = w.n**3 * esz
    del c_d, g_d, h_d, ws

    hbm, src = peaks()
    achieved = prof["step_bytes"] / (prof["step_ms"] / 1e3) / 1e9 if prof["step_ms"] > 0 else None
    launch_ms = prof["step_ms"] / max(prof["step_launches"], 1)
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, steps, el, cores = oracle_sample(w, seconds_target=args.ref_seconds)
        # and on one core, a shorter sample
        import oracle.oracle as o
        o.set_num_threads(1)
        try:
            v1, steps1, el1, _ = oracle_sample(w, seconds_target=min(3.0, args.ref_seconds))
        finally:
            o.set_num_threads(cores)
        cpu = {"value": v, "unit": "voxel-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 CPU oracle wave operator W: {steps} leapfrog steps on the "
                         f"{w.n}^3 grid ({el:.1f} s)",
               "value_1core": v1,
               "sample_1core": f"the same on one core: {steps1} steps ({el1:.1f} s)"}
    bpp = {F.FP64: 32, F.FP32: 16, F.FP32_KAHAN: 28}[prob.precision]
    steps_per_pass = prof["steps"] / max(prof["step_launches"], 1)
    kernel = ("resident" if steps_per_pass > 2 else
              "two-step" if steps_per_pass > 1.5 else "single-step")
    common = {"traffic": NCU_TRAFFIC.get((args.workload, args.precision, kernel)),
              "traffic_source": "one ncu capture of the same kernel on the same grid (cold "
                                "caches), DRAM read + write bytes per launch",
              "steps_per_pass": steps_per_pass, "launch_ms": launch_ms,
              "launches_timed": prof["step_launches"], "steps_timed": prof["steps"]}
    rates = None if args.no_extras else guarded(fma_rates, F)
    if rates is not None and "error" in rates:
        rates = None
    if kernel == "resident" and args.precision in FLOP_PER_POINT_STEP:
        # the resident time loop (one launch per W): the state never leaves
        # the chip, so HBM is not its bound; report its arithmetic against
        # the measured FP32 FMA rate (else the rate derived from the clock)
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        if rates:
            peak, psrc = rates["fp32x2_tflops"], "measured: ffpat_debug_fma_rate (packed FP32)"
        else:
            peak = FP32_LANES * 2 * mhz * 1e6 / 1e12
            psrc = f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"
        flops = FLOP_PER_POINT_STEP[args.precision] * prof["steps"] * float(w.n) ** 3
        ach = flops / (prof["step_ms"] / 1e3) / 1e12 if prof["step_ms"] > 0 else None
        roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": (ach / peak) if ach else None, "peak_source": psrc,
                    "kernel": "resident time loop (k_wave_resident)",
                    "flop_per_point_step": FLOP_PER_POINT_STEP[args.precision],
                    "algorithmic_state_gbs": achieved, **common}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if achieved else None,
                    "peak_source": f"{src} hbm_gbs",
                    "kernel": ("two-step leapfrog pass (k_step2_kahan)" if kernel == "two-step"
                               else "leapfrog step"),
                    "bytes_per_point_pass": bpp, **common}
    line = {
        "metric": "voxel-steps/s", "value": value, "unit": "voxel-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {F.FP64: "f64", F.FP32: "f32", F.FP32_KAHAN: "f32"}[prob.precision],
        "data": "synthetic",
        "config": workload_config(w, wl, nt, F.PRECISION_NAMES[prob.precision], world),
        "fb_iters_per_s": world * args.steps / (dev_ms / 1e3),
        "wall_s": wall,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": world * vs_per_iter / e2e_s, "unit": "voxel-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and not args.no_extras:
        # measured after the timed region; a failure here is recorded in the
        # line instead of costing it
        line["fma_rates"] = rates
        line["fp32_vs_fp64"] = guarded(extra_precision, F, dev, rates, args.extra_iters)
        pool = guarded(serving_pool, F, dev, args.pool)
        if isinstance(pool, list):
            line["serving"] = guarded(extra_serving, F, pool, args)
            line["serve_vs_fp64"] = guarded(extra_serve_vs_fp64, F, dev, pool[:args.fp64_pool],
                                            args)
        else:
            line["serving"] = line["serve_vs_fp64"] = pool
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def guarded(fn, *a):
    """fn(*a), or {"error": ...} if it raises (for the optional keys of the line)."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def fma_rates(F):
    """Measured FMA rates of the FP64, FP32 and packed FP32 pipes (TFLOP/s)."""
    return {"fp64_tflops": F.debug_fma_rate(F.FMA_FP64) / 1e12,
            "fp32_tflops": F.debug_fma_rate(F.FMA_FP32) / 1e12,
            "fp32x2_tflops": F.debug_fma_rate(F.FMA_FP32X2) / 1e12,
            "how": "ffpat_debug_fma_rate: every SM full, 8 independent FMA chains per thread, "
                   "best of 3 launches, CUDA events"}


def extra_precision(F, dev, rates, iters):
    """The 128^3 solve (90 angles, T = 1.2, identity Lambda) in FP64, FP32 and
    FP32-Kahan with the same step from h = 0: milliseconds per FB iteration
    (CUDA events, after one warm-up iteration), the relative L2 difference of
    each FP32 iterate from the FP64 GPU iterate after `iters` iterations, and
    the FP64 leapfrog's use of the FP64 pipe against its measured FMA rate."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300.inputs import add_noise, config
    w = config(2)
    p64 = F.problem(w.n, w.T, w.n_angles, F.FP64)
    c64 = torch.as_tensor(w.c, device=dev)
    g64 = F.forward(p64, c64, torch.as_tensor(w.h, device=dev))
    gd = torch.as_tensor(add_noise(g64.cpu().numpy(), w.noise, w.noise_rel), device=dev)
    step = 1.0 / F.opnorm(p64, c64, torch.ones_like(c64), iters=20)
    nt, _, _ = F.problem_info(p64, float(w.c.max()))
    out = {"workload": "single solve N=128^3, 90 angles, T=1.2, identity Lambda", "nt": nt,
           "iters": iters, "step": step}
    res = {}
    for name, prec in (("fp64", F.FP64), ("fp32", F.FP32), ("fp32-kahan", F.FP32_KAHAN)):
        prob = F.problem(w.n, w.T, w.n_angles, prec)
        dt = F.torch_dtype(prob)
        c, g = c64.to(dt), gd.to(dt)
        ws = F.workspace(prob, dev)
        F.fb_solve(prob, c, g, w.lam, step, 1, ws=ws, history=False)
        torch.cuda.synchronize()
        F.profile_enable(True)
        F.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h, _, _ = F.fb_solve(prob, c, g, w.lam, step, iters, ws=ws, history=False)
        e1.record()
        torch.cuda.synchronize()
        prof = F.profile_read()
        F.profile_enable(False)
        res[name] = (h.double(), e0.elapsed_time(e1) / iters, prof)
        del ws
    ref = res["fp64"][0]
    for name, (h, ms, prof) in res.items():
        out[name] = {"ms_per_fb_iter": ms,
                     "voxel_steps_per_s": 2.0 * nt * w.n ** 3 / (ms / 1e3),
                     "rel_l2_vs_fp64_gpu": float((h - ref).norm() / ref.norm()),
                     "speedup_vs_fp64": res["fp64"][1] / ms}
    prof = res["fp64"][2]
    if prof["steps"] and rates:
        rate = prof["steps"] * float(w.n) ** 3 / (prof["step_ms"] / 1e3)
        ops = FP64_OPS_PER_POINT_STEP * rate
        # the probe counts 2 FLOP per DFMA: its instruction rate is half its FLOP rate
        peak_ops = rates["fp64_tflops"] * 1e12 / 2
        out["fp64_leapfrog"] = {"point_steps_per_s": rate, "us_per_step":
                                1e3 * prof["step_ms"] / prof["steps"],
                                "fp64_ops_per_point_step": FP64_OPS_PER_POINT_STEP,
                                "fp64_pipe_frac": ops / peak_ops, "bound": "fp64 alu",
                                "peak_source": "measured: ffpat_debug_fma_rate (FP64)"}
    return out


def serving_pool(F, dev, count):
    """`count` requests of the serving mix (sizes from {64, 96, 128, 192}^3,
    45 / 90 / 180 angles, T in [0.8, 1.4], 20-60 iterations, each from its own
    seed): FP64 sound speed, FP64 data (library FP64 forward + 1 % noise) and
    the step 1/L from 20 power iterations of the FP32-Kahan operator."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300.inputs import add_noise, config
    pool = []
    for s in range(1, count + 1):
        w = config(4, seed=1000 + s)
        p32 = F.problem(w.n, w.T, w.n_angles, F.FP32_KAHAN)
        p64 = F.problem(w.n, w.T, w.n_angles, F.FP64)
        c64 = torch.as_tensor(w.c, device=dev)
        g64 = F.forward(p64, c64, torch.as_tensor(w.h, device=dev))
        gd = add_noise(g64.cpu().numpy(), w.noise, w.noise_rel)
        c32 = c64.float()
        step = 1.0 / F.opnorm(p32, c32, torch.ones_like(c32), iters=20)
        nt, _, _ = F.problem_info(p32, float(w.c.astype(np.float32).max()))
        pool.append(dict(p32=p32, p64=p64, c=w.c, g=gd, step=step, iters=w.iters, nt=nt,
                         n=w.n, nth=w.n_angles))
    torch.cuda.synchronize()
    return pool


def extra_serving(F, pool, args):
    """Poisson arrivals (rate args.rate) over args.window seconds, cycling the
    pool, through the continuous-batching server; then drained."""
    import numpy as np
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=100000))
    arrivals = arrivals[arrivals < args.window]
    budget = int(args.budget_gb * (1 << 30))
    tickets = []
    with F.Server(budget, args.slots) as srv, Clocks(0) as clk:
        t0 = time.perf_counter()
        k = 0
        while k < len(arrivals) or any(t is not None for t in tickets):
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                r = pool[k % len(pool)]
                tickets.append(srv.submit(r["p32"], r["c"].astype(np.float32),
                                          r["g"].astype(np.float32), 1e-3, r["step"],
                                          r["iters"]))
                k += 1
            for i, t in enumerate(tickets):
                if t is not None and srv.poll(t) is not None:
                    tickets[i] = None
            time.sleep(0.001)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
    return {"recons_per_s": st["completed"] / elapsed, "p50_ms": st["p50_ms"],
            "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
            "completed": st["completed"], "failed": st["failed"], "window_s": args.window,
            "elapsed_s": elapsed, "arrival_rate_per_s": args.rate,
            "voxel_steps_per_s": st["point_steps"] / elapsed, "ticks": st["ticks"],
            "pool": len(pool), "slots": args.slots, "precision": "fp32-kahan",
            "requests": [{"n": r["n"], "angles": r["nth"], "iters": r["iters"]} for r in pool],
            "clocks": clk.summary()}


def extra_serve_vs_fp64(F, dev, pool, args):
    """The served FP32 path against the plain FP64 GPU path on the same
    requests: the pool as one burst through the server (FP32-Kahan, all
    submitted at once) and the same reconstructions one after another through
    ffpat_fb_solve in FP64, same step and iteration count; recons/s of both,
    their ratio and the largest relative L2 difference of a served image from
    its FP64 reconstruction."""
    import numpy as np
    import torch
    budget = int(args.budget_gb * (1 << 30))
    served = {}
    with F.Server(budget, args.slots) as srv:
        r = pool[0]
        srv.wait(srv.submit(r["p32"], r["c"].astype(np.float32), r["g"].astype(np.float32),
                            1e-3, r["step"], 1))
        t0 = time.perf_counter()
        tickets = [(i, srv.submit(r["p32"], r["c"].astype(np.float32),
                                  r["g"].astype(np.float32), 1e-3, r["step"], r["iters"]))
                   for i, r in enumerate(pool)]
        for i, t in tickets:
            served[i] = srv.wait(t)[0]
        t_served = time.perf_counter() - t0
    t64, errs = 0.0, []
    for i, r in enumerate(pool):
        c_d = torch.as_tensor(r["c"], device=dev)
        g_d = torch.as_tensor(r["g"], device=dev)
        ws = F.workspace(r["p64"], dev)
        torch.cuda.synchronize()
        a = time.perf_counter()
        h64, _, _ = F.fb_solve(r["p64"], c_d, g_d, 1e-3, r["step"], r["iters"], ws=ws,
                               history=False)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - a
        h64 = h64.cpu().numpy()
        h32 = np.asarray(served[i], dtype=np.float64)
        errs.append(float(np.linalg.norm(h32 - h64) / np.linalg.norm(h64)))
        del ws
    r_served, r64 = len(pool) / t_served, len(pool) / t64
    return {"served_fp32_kahan_recons_per_s": r_served, "plain_fp64_gpu_recons_per_s": r64,
            "ratio": r_served / r64, "max_rel_l2_vs_fp64": max(errs), "rel_l2_vs_fp64": errs,
            "pool": len(pool),
            "how": "pool served as one burst (FP32-Kahan) vs ffpat_fb_solve in FP64 one "
                   "request after another, same step and iterations, wall time"}


def run_serve(args):
    """Serving mix (Poisson arrivals of requests of mixed size) through the
    continuous-batching server; prints one JSON line with recons/s and p50/p99."""
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    build_lib.build()
    F.lib()
    dev = torch.device("cuda", 0)
    res = extra_serving(F, serving_pool(F, dev, args.pool), args)
    print(json.dumps({"mode": "serve", "metric": "recons/s", "value": res["recons_per_s"],
                      "unit": "recons/s", "n_gpus": 1, "higher_is_better": True, **res,
                      "config": {"workload": "serving mix: N in {64,96,128,192}, 45/90/180 "
                                             "angles, T in [0.8,1.4], 20-60 FB iterations, "
                                             "FP32-Kahan", "budget_gb": args.budget_gb},
                      "dtype": "f32", "data": "synthetic"}))
    return 0


def run_serve_vs_fp64(args):
    """The served FP32 path against the plain FP64 GPU path on the same
    requests (see extra_serve_vs_fp64); prints one JSON line."""
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    build_lib.build()
    F.lib()
    dev = torch.device("cuda", 0)
    pool = serving_pool(F, dev, args.pool)
    res = extra_serve_vs_fp64(F, dev, pool, args)
    print(json.dumps({"mode": "serve_vs_fp64", "metric": "recons/s", "unit": "recons/s", **res,
                      "requests": [{"n": r["n"], "iters": r["iters"]} for r in pool],
                      "config": {"workload": "serving pool: N in {64,96,128,192}, 45/90/180 "
                                             "angles, T in [0.8,1.4], 20-60 FB iterations; "
                                             "FP32-Kahan served as one burst vs FP64 "
                                             "ffpat_fb_solve one after another",
                                 "pool": args.pool, "slots": args.slots},
                      "dtype": "f32 vs f64", "data": "synthetic"}))
    return 0


def run_op(args):
    """One library operation on a seeded random problem, timed with CUDA
    events: the driver for timing and profiling single kernels.  --op-steps
    sets T so that the wave operator takes exactly that many leapfrog steps
    (c in [0.75, 1.4], cfl 0.3); --path picks the leapfrog kernel."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F

    build_lib.build()
    F.set_stencil_path(args.path)
    prec = {"fp64": F.FP64, "fp32": F.FP32, "fp32-kahan": F.FP32_KAHAN}[args.precision]
    n = args.n
    cmax = 1.4
    T = args.op_steps * 0.3 * (2.0 / n) / cmax * (1 - 1e-9)
    prob = F.problem(n, T, args.angles, prec, precond=1 if (args.op == "ramp" or args.ramp) else 0)
    nt, _, _ = F.problem_info(prob, cmax)
    dt = F.torch_dtype(prob)
    gen = torch.Generator(device="cuda").manual_seed(args.seed)
    c = (0.75 + 0.65 * torch.rand((n, n, n), generator=gen, device="cuda", dtype=torch.float64))
    c.view(-1)[0] = cmax
    c = c.to(dt)
    h = torch.randn((n, n, n), generator=gen, device="cuda", dtype=torch.float64).to(dt)
    g = torch.randn((args.angles, n, n), generator=gen, device="cuda",
                    dtype=torch.float64).to(dt)
    ws = F.workspace(prob)
    out_v = torch.empty_like(h)
    out_d = torch.empty_like(g)

    def run():
        if args.op == "wave":
            F.wave(prob, c, h, out_v, ws=ws)
        elif args.op == "wave_t":
            F.wave(prob, c, h, out_v, transpose=True, ws=ws)
        elif args.op == "forward":
            F.forward(prob, c, h, out_d, ws=ws)
        elif args.op == "adjoint":
            F.adjoint(prob, c, g, out_v, ws=ws)
        elif args.op == "project":
            F.project(prob, h, out_d)
        elif args.op == "backproject":
            F.backproject(prob, g, out_v)
        elif args.op == "ramp":
            F.ramp(prob, g, out_d)
        elif args.op == "fb":
            F.fb_solve(prob, c, g, 1e-3, 1e-3, 1, h=out_v.zero_(), ws=ws, history=False)

    run()
    torch.cuda.synchronize()
    F.profile_enable(True)
    F.profile_read()
    times = []
    for _ in range(args.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.inner):
            run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / args.inner)
    prof = F.profile_read()
    F.profile_enable(False)
    res = {"mode": "op", "op": args.op, "path": args.path, "n": n, "angles": args.angles,
           "nt": nt, "precision": args.precision, "ms": times, "ms_min": min(times)}
    if prof["step_launches"]:
        res["step_ms_avg"] = prof["step_ms"] / prof["step_launches"]
        res["step_gbs"] = prof["step_bytes"] / (prof["step_ms"] / 1e3) / 1e9
        res["voxel_steps_per_s"] = prof["steps"] * n**3 / (prof["step_ms"] / 1e3)
        res["step_ms_per_step"] = prof["step_ms"] / max(prof["steps"], 1)
    assert np.isfinite(out_v.double().sum().item()) or args.op in ("forward", "project", "ramp")
    print(json.dumps(res))
    return 0


def run_precision(args):
    """FP64 vs FP32 vs FP32-Kahan on the 128^3 single solve: time per FB
    iteration and the relative L2 difference of the iterate from the FP64 GPU
    iterate after the same number of iterations; and the relative L2
    difference of one W application (1344 leapfrog steps) on the 384^3
    workload from the FP64 GPU result."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise, config

    build_lib.build()
    dev = torch.device("cuda", 0)
    w = config(2)
    p64 = F.problem(w.n, w.T, w.n_angles, F.FP64)
    c64 = torch.as_tensor(w.c, device=dev)
    g64 = F.forward(p64, c64, torch.as_tensor(w.h, device=dev))
    gd = torch.as_tensor(add_noise(g64.cpu().numpy(), w.noise, w.noise_rel), device=dev)
    step = 1.0 / F.opnorm(p64, c64, torch.ones_like(c64), iters=20)
    res = {}
    for name, prec in (("fp64", F.FP64), ("fp32", F.FP32), ("fp32-kahan", F.FP32_KAHAN)):
        prob = F.problem(w.n, w.T, w.n_angles, prec)
        dt = F.torch_dtype(prob)
        c, g = c64.to(dt), gd.to(dt)
        F.fb_solve(prob, c, g, w.lam, step, 1, history=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h, st, _ = F.fb_solve(prob, c, g, w.lam, step, args.iters, history=False)
        e1.record()
        torch.cuda.synchronize()
        res[name] = (h.double(), e0.elapsed_time(e1) / args.iters)
    ref = res["fp64"][0]
    out = {"mode": "precision", "workload": "single solve N=128^3, 90 angles, T=1.2",
           "iters": args.iters, "step": step}
    for name, (h, ms) in res.items():
        out[name] = {"ms_per_fb_iter": ms,
                     "rel_l2_vs_fp64_gpu": float((h - ref).norm() / ref.norm()),
                     "speedup_vs_fp64": res["fp64"][1] / ms}
    # one application of W on the long 384^3 workload (1344 steps), where the
    # rounding of the FP32 forms accumulates longest
    w5 = config(5)
    waves = {}
    for name, prec in (("fp64", F.FP64), ("fp32", F.FP32), ("fp32-kahan", F.FP32_KAHAN)):
        prob = F.problem(w5.n, w5.T, w5.n_angles, prec)
        dt = F.torch_dtype(prob)
        c5 = torch.as_tensor(w5.c, device=dev).to(dt)
        h5 = torch.as_tensor(w5.h, device=dev).to(dt)
        waves[name] = F.wave(prob, c5, h5).double()
        del c5, h5
        torch.cuda.synchronize()
    r5 = waves["fp64"]
    nt5, _, _ = F.problem_info(F.problem(w5.n, w5.T, w5.n_angles), float(w5.c.max()))
    out["wave_384"] = {"nt": nt5, **{name: float((v - r5).norm() / r5.norm())
                                     for name, v in waves.items() if name != "fp64"}}
    print(json.dumps(out))
    return 0


# FP32 FFMA peak of the GB300 for the dense DCT passes of the gradient prox:
# 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz (maximum SM clock)
FP32_FFMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def run_paper(args):
    """The paper's experimental setting (Sec. 5) in 3D: the source box N^3 on
    [-1, 1]^3, the wave grid padded to [-3, 3]^3 (pad = N, the paper's 3x
    domain), T = 2, data only where |xi| > 1 (the rays that miss the source
    box), 10 % relative noise, R = 1/2 |grad h|^2 with s lambda / dx^2 = 1 and
    s = 1/L; the one-step method (Algorithm 8, ramp-preconditioned) against the two-step method
    (Algorithm 9): time per iteration, voxel-steps/s on the wave grid, the
    gradient prox's own rate, and the relative L2 error of both reconstructions
    after the same number of iterations.  The phantom and sound speed are the
    synthetic 20-ball / Gaussian-random-field pair (the paper's are not
    published), so the errors are context, not a reproduction."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise, config, extend_speed, padded_axis

    build_lib.build()
    dev = torch.device("cuda", 0)
    n, pad, T, nth = args.paper_n, args.paper_n, 2.0, args.paper_angles
    nw = n + 2 * pad
    w = config(2, n=n)
    c_np = extend_speed(w.c, pad)
    prec = {"fp32-kahan": F.FP32_KAHAN, "fp32": F.FP32, "fp64": F.FP64}[args.precision]
    # Algorithm 8 is the preconditioned one-step method: Lambda = ramp filter
    prob = F.problem(n, T, nth, prec, F.PRECOND_RAMP, pad=pad)
    dt = F.torch_dtype(prob)
    p64 = F.problem(n, T, nth, F.FP64, pad=pad)
    g64 = F.forward(p64, torch.as_tensor(c_np, device=dev), torch.as_tensor(w.h, device=dev))
    rng = np.random.default_rng(1901)
    mask_np = np.broadcast_to((np.abs(padded_axis(n, pad)) > 1.0).astype(np.float64),
                              (nth, nw, nw)).copy()
    g_np = mask_np * add_noise(g64.cpu().numpy(), rng.standard_normal((nth, nw, nw)), 0.10)
    del g64
    c = torch.as_tensor(c_np, device=dev).to(dt)
    g = torch.as_tensor(g_np, device=dev).to(dt)
    mask = torch.as_tensor(mask_np, device=dev).to(dt)
    h_true = torch.as_tensor(w.h, device=dev)
    ws = F.workspace(prob, dev)
    dx = 2.0 / n
    nt, _, _ = F.problem_info(prob, float(c.double().max()))
    iters = args.iters

    def err(h):
        return float((h.double() - h_true).norm() / h_true.norm())

    out = {"mode": "paper",
           "workload": f"source box {n}^3 on [-1,1]^3, wave grid {nw}^3 on [-3,3]^3, T = 2, "
                       f"{nth} angles, data for |xi| > 1, 10% noise, R = 1/2|grad h|^2",
           "precision": F.PRECISION_NAMES[prec], "nt": nt, "iters": iters}
    # one-step: step 1/L of the masked A^T A, then lambda with s lambda / dx^2 = 1
    _, st0, _ = F.fb_solve_masked(prob, c, g, 0.0, 0.0, 0, mask=mask, ws=ws, reg=F.REG_GRAD2)
    s1 = st0["step"]
    lam1 = dx * dx / s1
    F.fb_solve_masked(prob, c, g, lam1, s1, 1, mask=mask, ws=ws, reg=F.REG_GRAD2, history=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h1, st1, _ = F.fb_solve_masked(prob, c, g, lam1, s1, iters, mask=mask, ws=ws,
                                   reg=F.REG_GRAD2, history=False)
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / iters
    vs = 2.0 * nt * float(nw) ** 3
    out["one_step"] = {"ms_per_iter": ms1, "voxel_steps_per_s": vs / (ms1 / 1e3),
                       "rel_l2_error": err(h1), "step": s1, "lambda": lam1,
                       "objective": st1["objective"]}
    # two-step: X^{-1} of the masked data, then FB on 1/2 ||W h - g~||^2
    _, st0, _ = F.fb_two_step(prob, c, g, 0.0, 0.0, 0, ws=ws, reg=F.REG_GRAD2)
    s2 = st0["step"]
    lam2 = dx * dx / s2
    torch.cuda.synchronize()
    e0.record()
    h2, st2, _ = F.fb_two_step(prob, c, g, lam2, s2, iters, ws=ws, reg=F.REG_GRAD2, history=False)
    e1.record()
    torch.cuda.synchronize()
    ms2 = e0.elapsed_time(e1) / iters
    out["two_step"] = {"ms_per_iter": ms2, "voxel_steps_per_s": vs / (ms2 / 1e3),
                       "rel_l2_error": err(h2), "step": s2, "lambda": lam2}
    # the gradient prox alone (six DCT passes on the box, 2 n^4 FLOP each)
    f = torch.randn((n, n, n), device=dev, dtype=torch.float64).to(dt)
    F.prox_grad(prob, f, 1.0, ws=ws)
    torch.cuda.synchronize()
    reps = 20
    e0.record()
    for _ in range(reps):
        F.prox_grad(prob, f, 1.0, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1) / reps
    flop = 6 * 2.0 * float(n) ** 4
    out["prox"] = {"ms": pms, "tflops": flop / (pms / 1e3) / 1e12, "bound": "alu",
                   "peak_tflops": FP32_FFMA_TFLOPS if prec != F.FP64 else None,
                   "share_of_one_step_iter": pms / ms1}
    print(json.dumps(out))
    return 0


def run_grad(args):
    """The differentiable operator on the 192^3 workload (FP32, 90 angles,
    T = 1): loss 1/2 |A(h, c) - g|^2 through torch.autograd, gradients for h
    and c (wavefield checkpoints every 16 steps, each segment recomputed in
    the backward pass), and for h alone (the adjoint).  Reports milliseconds
    per forward + backward and the voxel-steps they run (forward Nt steps;
    backward Nt recomputed plus Nt transposed steps when c needs a gradient,
    Nt transposed steps for h alone)."""
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.autograd import forward_op
    from paper_1901_06503_gb300.inputs import config

    build_lib.build()
    dev = torch.device("cuda", 0)
    w = config(3)
    prob = F.problem(w.n, w.T, w.n_angles, F.FP32)
    c0 = torch.as_tensor(w.c, device=dev).float()
    h0 = torch.as_tensor(w.h, device=dev).float()
    nt, _, _ = F.problem_info(prob, float(c0.double().max()))
    g = (F.forward(prob, c0, h0) * 1.01).detach()
    reps = max(1, args.iters)
    out = {"mode": "grad", "workload": w.name, "n": w.n, "nt": nt, "every": 16,
           "precision": "fp32", "reps": reps}
    for name, want_c in (("grad_h_and_c", True), ("grad_h", False)):
        h = h0.clone().requires_grad_(True)
        c = c0.clone().requires_grad_(want_c)

        def step():
            loss = 0.5 * ((forward_op(h, c, prob, 16) - g) ** 2).sum()
            loss.backward()
            return loss

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            h.grad = None
            c.grad = None
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        steps = nt * (3 if want_c else 2)
        out[name] = {"ms_per_forward_backward": ms, "wave_steps": steps,
                     "voxel_steps_per_s": steps * float(w.n) ** 3 / (ms / 1e3)}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg5")
    ap.add_argument("--precision", choices=["fp32-kahan", "fp32", "fp64"], default="fp32-kahan")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="fb: leave out the FP32-vs-FP64, FMA-rate and serving keys")
    ap.add_argument("--mode", choices=["fb", "op", "serve", "serve_vs_fp64", "precision",
                                       "paper", "grad"],
                    default="fb",
                    help="fb: the default FB-iteration line; op: one library operation "
                         "(kernel timing and profiling); serve: the serving mix; "
                         "precision: FP64 vs FP32 vs FP32-Kahan on the 128^3 solve; "
                         "paper: the paper's experimental setting in 3D (one- vs two-step); "
                         "serve_vs_fp64: served FP32 burst vs plain FP64 GPU solves; "
                         "grad: forward + backward of the differentiable 192^3 operator")
    ap.add_argument("--paper-n", type=int, default=64, help="paper: source box points per axis")
    ap.add_argument("--paper-angles", type=int, default=180, help="paper: projection angles")
    ap.add_argument("--window", type=float, default=10.0, help="serve: arrival window (s)")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: Poisson arrival rate (1/s)")
    ap.add_argument("--pool", type=int, default=8, help="serve: distinct requests cycled")
    ap.add_argument("--fp64-pool", type=int, default=6,
                    help="fb extras: requests of the pool solved in FP64 for the comparison")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--iters", type=int, default=20, help="precision / paper: FB iterations")
    ap.add_argument("--extra-iters", type=int, default=100,
                    help="fb extras: FB iterations of the FP32-vs-FP64 comparison (128^3)")
    # --mode op
    ap.add_argument("--op", choices=["wave", "wave_t", "forward", "adjoint", "project",
                                     "backproject", "ramp", "fb"], default="wave")
    ap.add_argument("--n", type=int, default=128, help="op: grid points per axis")
    ap.add_argument("--angles", type=int, default=90, help="op: projection angles")
    ap.add_argument("--op-steps", type=int, default=16, help="op: leapfrog steps of W")
    ap.add_argument("--repeat", type=int, default=3, help="op: timed repetitions")
    ap.add_argument("--inner", type=int, default=1,
                    help="op: calls per timed repetition (ms is per call; for short kernels)")
    ap.add_argument("--seed", type=int, default=0, help="op: random seed")
    ap.add_argument("--ramp", action="store_true", help="op: ramp preconditioner (Lambda)")
    ap.add_argument("--path", type=int, default=0,
                    help="op: leapfrog kernel: 0 auto, 1 plain, 2 TMA, 3 two-step, 4 resident")
    args = ap.parse_args()
    if args.mode == "op":
        return run_op(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "serve_vs_fp64":
        return run_serve_vs_fp64(args)
    if args.mode == "grad":
        return run_grad(args)
    if args.mode == "paper":
        return run_paper(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
