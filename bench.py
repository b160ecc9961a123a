"""Benchmark of the hot path: iterations of Algorithm 8 (one-step FB) on the
single-instance 128^3 workload (90 angles, T = 1.2, FP32-Kahan wavefields).

One step = one FB iteration = W (333 leapfrog steps) + P + residual + P^T +
W^T (333 steps) + the fused prox update with FP64 norms.  The metric is
voxel-steps per second (2 Nt N^3 per iteration over the device time), with
FB iterations per second alongside.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cfg2|cfg5|cfg1] [--precision fp32-kahan|fp32|fp64]

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

# DRAM bytes per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, cold caches): the single-step
# kernel at 128^3 (profiles/k_step_tma_fp32kahan_n128.md) and the two-step
# kernel at 384^3 (profiles/k_step2_kahan_fp32kahan_n384.md).  Keyed by
# (workload, precision); None where no capture of the current kernel exists.
# DRAM bytes per launch of the dominant kernel, from one ncu capture each
# (profiles/): the step pass of the 384^3 workload; at 128^3 the resident time
# loop, whose DRAM traffic is its first load of p^0 and kap / 12 (the state
# stays on chip, so it does not grow with the step count)
NCU_TRAFFIC = {("cfg2", "fp32-kahan"): 17.167104e6, ("cfg5", "fp32-kahan"): 1544.95488e6}

# algorithmic FP32 operations per point-step of the difference-form update:
# 12 subtractions, 10 additions and one FMA (2) for 12 h^2 L4 p, then the
# Kahan increment (FMA + 4 adds) or the three-term update (FMA + 2 adds)
FLOP_PER_POINT_STEP = {"fp32-kahan": 30, "fp32": 28}
# FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop (FMA) per clock
FP32_LANES = 152 * 128

WORKLOADS = {
    "cfg2": dict(cfg=2, label="single solve N=128^3, 90 angles, T=1.2, 20 balls, GRF sound speed"),
    "cfg5": dict(cfg=5, label="large solve N=384^3, 180 angles, T=1.5, ramp-preconditioned"),
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


def make_problem(args):
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import config
    wl = WORKLOADS[args.workload]
    w = config(wl["cfg"])
    prec = {"fp32-kahan": F.FP32_KAHAN, "fp32": F.FP32, "fp64": F.FP64}[args.precision]
    prob = F.problem(w.n, w.T, w.n_angles, prec, w.precond)
    return w, wl, prob


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
        "config": {"workload": wl["label"], "n": w.n, "n_angles": w.n_angles, "T": w.T},
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
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    dev_ms = max_over_ranks(dev_ms, world, dev)
    vs_per_iter = 2.0 * nt * float(w.n) ** 3
    value = world * args.steps * vs_per_iter / (dev_ms / 1e3)
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
    common = {"traffic": NCU_TRAFFIC.get((args.workload, args.precision)),
              "traffic_source": "ncu capture of the same kernel (cold caches), DRAM bytes per launch",
              "steps_per_pass": steps_per_pass, "launch_ms": launch_ms,
              "launches_timed": prof["step_launches"], "steps_timed": prof["steps"]}
    if steps_per_pass > 2 and args.precision in FLOP_PER_POINT_STEP:
        # the resident time loop (one launch per W): the state never leaves
        # the chip, so HBM is not its bound; report its arithmetic against
        # the FP32 CUDA-core peak at the maximum SM clock
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = FP32_LANES * 2 * mhz * 1e6 / 1e12
        flops = FLOP_PER_POINT_STEP[args.precision] * prof["steps"] * float(w.n) ** 3
        ach = flops / (prof["step_ms"] / 1e3) / 1e12 if prof["step_ms"] > 0 else None
        roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": (ach / peak) if ach else None,
                    "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz",
                    "kernel": "resident time loop (k_wave_resident)",
                    "flop_per_point_step": FLOP_PER_POINT_STEP[args.precision],
                    "algorithmic_state_gbs": achieved, **common}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if achieved else None,
                    "peak_source": f"{src} hbm_gbs", "kernel": "leapfrog pass",
                    "bytes_per_point_pass": bpp, **common}
    line = {
        "metric": "voxel-steps/s", "value": value, "unit": "voxel-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {F.FP64: "f64", F.FP32: "f32", F.FP32_KAHAN: "f32"}[prob.precision],
        "data": "synthetic",
        "config": {"workload": wl["label"], "n": w.n, "n_angles": w.n_angles, "T": w.T,
                   "nt": nt, "precision": F.PRECISION_NAMES[prob.precision],
                   "fb_iteration": "W + P + residual + P^T + W^T + prox update",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "fb_iters_per_s": world * args.steps / (dev_ms / 1e3),
        "wall_s": wall,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": world * vs_per_iter / e2e_s, "unit": "voxel-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Serving mix (Poisson arrivals of requests of mixed size) through the
    continuous-batching server; prints one JSON line with recons/s and p50/p99."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise, config

    build_lib.build()
    F.lib()
    dev = torch.device("cuda", 0)
    pool = []
    for s in range(1, args.pool + 1):
        w = config(4, seed=1000 + s)
        prob = F.problem(w.n, w.T, w.n_angles, F.FP32_KAHAN)
        c = torch.as_tensor(w.c, device=dev).float()
        g = F.forward(prob, c, torch.as_tensor(w.h, device=dev).float())
        gd = add_noise(g.double().cpu().numpy(), w.noise, w.noise_rel).astype(np.float32)
        step = 1.0 / F.opnorm(prob, c, torch.ones_like(c), iters=20)
        nt, _, _ = F.problem_info(prob, float(w.c.astype(np.float32).max()))
        pool.append((prob, w.c.astype(np.float32), gd, step, w.iters, nt, w.n))
    torch.cuda.synchronize()
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
                prob, c, gd, step, iters, nt, n = pool[k % len(pool)]
                tickets.append(srv.submit(prob, c, gd, 1e-3, step, iters))
                k += 1
            for i, t in enumerate(tickets):
                if t is not None and srv.poll(t) is not None:
                    tickets[i] = None
            time.sleep(0.001)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
    ps = st["point_steps"]
    line = {"mode": "serve", "metric": "recons/s", "value": st["completed"] / elapsed,
            "unit": "recons/s", "n_gpus": 1, "higher_is_better": True,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "max_ms": st["max_ms"], "completed": st["completed"], "failed": st["failed"],
            "window_s": args.window, "elapsed_s": elapsed, "arrival_rate": args.rate,
            "voxel_steps_per_s": ps / elapsed, "ticks": st["ticks"],
            "config": {"workload": "serving mix: N in {64,96,128,192}, 45/90/180 angles, "
                                   "T in [0.8,1.4], 20-60 FB iterations, FP32-Kahan",
                       "pool": args.pool, "slots": args.slots, "budget_gb": args.budget_gb},
            "clocks": clk.summary(), "dtype": "f32", "data": "synthetic"}
    print(json.dumps(line))
    return 0


def run_serve_vs_fp64(args):
    """The served FP32 path against the plain FP64 GPU path on the same
    requests: a burst of the serving pool through the continuous-batching
    server (FP32-Kahan, all submitted at once: saturated throughput) and the
    same reconstructions one after another through ffpat_fb_solve in FP64,
    with the same step and iteration count.  Prints recons/s of both, their
    ratio and the largest relative L2 difference of a served image from its
    FP64 reconstruction."""
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise, config

    build_lib.build()
    F.lib()
    dev = torch.device("cuda", 0)
    pool = []
    for s in range(1, args.pool + 1):
        w = config(4, seed=1000 + s)
        p32 = F.problem(w.n, w.T, w.n_angles, F.FP32_KAHAN)
        p64 = F.problem(w.n, w.T, w.n_angles, F.FP64)
        c64 = torch.as_tensor(w.c, device=dev)
        g64 = F.forward(p64, c64, torch.as_tensor(w.h, device=dev))
        gd = add_noise(g64.cpu().numpy(), w.noise, w.noise_rel)
        step = 1.0 / F.opnorm(p64, c64, torch.ones_like(c64), iters=20)
        pool.append((p32, p64, w.c, gd, step, w.iters, w.n))
    torch.cuda.synchronize()
    budget = int(args.budget_gb * (1 << 30))
    served = {}
    with F.Server(budget, args.slots) as srv:
        # warm-up: one request through the server
        p32, _, c, gd, step, iters, _ = pool[0]
        srv.wait(srv.submit(p32, c.astype(np.float32), gd.astype(np.float32), 1e-3, step, 1))
        t0 = time.perf_counter()
        tickets = [(i, srv.submit(p32, c.astype(np.float32), gd.astype(np.float32), 1e-3, step,
                                  iters))
                   for i, (p32, _, c, gd, step, iters, _) in enumerate(pool)]
        for i, t in tickets:
            served[i] = srv.wait(t)[0]
        t_served = time.perf_counter() - t0
    # FP64, one reconstruction after another (device-resident inputs)
    t64 = 0.0
    errs = []
    for i, (_, p64, c, gd, step, iters, _) in enumerate(pool):
        c_d = torch.as_tensor(c, device=dev)
        g_d = torch.as_tensor(gd, device=dev)
        ws = F.workspace(p64, dev)
        torch.cuda.synchronize()
        a = time.perf_counter()
        h64, _, _ = F.fb_solve(p64, c_d, g_d, 1e-3, step, iters, ws=ws, history=False)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - a
        h64 = h64.cpu().numpy()
        h32 = np.asarray(served[i], dtype=np.float64)
        errs.append(float(np.linalg.norm(h32 - h64) / np.linalg.norm(h64)))
        del ws
    r_served = len(pool) / t_served
    r64 = len(pool) / t64
    line = {"mode": "serve_vs_fp64", "metric": "recons/s", "unit": "recons/s",
            "served_fp32_kahan": r_served, "plain_fp64_gpu": r64, "ratio": r_served / r64,
            "max_rel_l2_vs_fp64": max(errs), "rel_l2_vs_fp64": errs,
            "requests": [{"n": n, "iters": it} for (_, _, _, _, _, it, n) in pool],
            "config": {"workload": "serving pool: N in {64,96,128,192}, 45/90/180 angles, "
                                   "T in [0.8,1.4], 20-60 FB iterations; FP32-Kahan served as "
                                   "one burst vs FP64 ffpat_fb_solve one after another",
                       "pool": args.pool, "slots": args.slots},
            "dtype": "f32 vs f64", "data": "synthetic"}
    print(json.dumps(line))
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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg2")
    ap.add_argument("--precision", choices=["fp32-kahan", "fp32", "fp64"], default="fp32-kahan")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["fb", "serve", "serve_vs_fp64", "precision", "paper",
                                       "grad"],
                    default="fb",
                    help="fb: the default FB-iteration line; serve: the serving mix; "
                         "precision: FP64 vs FP32 vs FP32-Kahan on the 128^3 solve; "
                         "paper: the paper's experimental setting in 3D (one- vs two-step); "
                         "serve_vs_fp64: served FP32 burst vs plain FP64 GPU solves; "
                         "grad: forward + backward of the differentiable 192^3 operator")
    ap.add_argument("--paper-n", type=int, default=64, help="paper: source box points per axis")
    ap.add_argument("--paper-angles", type=int, default=180, help="paper: projection angles")
    ap.add_argument("--window", type=float, default=20.0, help="serve: arrival window (s)")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: Poisson arrival rate (1/s)")
    ap.add_argument("--pool", type=int, default=12, help="serve: distinct requests cycled")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--iters", type=int, default=20, help="precision / paper: FB iterations")
    args = ap.parse_args()
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
