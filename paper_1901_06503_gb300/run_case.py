"""Run one library operation on a seeded synthetic problem and report its
device time (CUDA events): a driver for timing and profiling single kernels.

  python -m paper_1901_06503_gb300.run_case --op wave --n 384 --steps 12 \
         --precision fp32-kahan --repeat 3

--steps sets T so that the wave operator takes exactly that many leapfrog
steps (c in [0.75, 1.4], cfl 0.3).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import numpy as np
    import torch

    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F

    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["wave", "wave_t", "forward", "adjoint", "project",
                                     "backproject", "ramp", "fb"], default="wave")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--angles", type=int, default=90)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32-kahan"], default="fp32-kahan")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--path", type=int, default=0, help="leapfrog kernel: 0 auto, 1 plain, 2 TMA, 3 two-step, 4 resident loop")
    a = ap.parse_args(argv)
    build_lib.build()
    F.set_stencil_path(a.path)
    prec = {"fp64": F.FP64, "fp32": F.FP32, "fp32-kahan": F.FP32_KAHAN}[a.precision]
    n = a.n
    cmax = 1.4
    T = a.steps * 0.3 * (2.0 / n) / cmax * (1 - 1e-9)
    prob = F.problem(n, T, a.angles, prec, precond=1 if a.op == "ramp" else 0)
    nt, _, _ = F.problem_info(prob, cmax)
    dt = F.torch_dtype(prob)
    gen = torch.Generator(device="cuda").manual_seed(a.seed)
    c = (0.75 + 0.65 * torch.rand((n, n, n), generator=gen, device="cuda", dtype=torch.float64))
    c.view(-1)[0] = cmax
    c = c.to(dt)
    h = torch.randn((n, n, n), generator=gen, device="cuda", dtype=torch.float64).to(dt)
    g = torch.randn((a.angles, n, n), generator=gen, device="cuda", dtype=torch.float64).to(dt)
    ws = F.workspace(prob)
    out_v = torch.empty_like(h)
    out_d = torch.empty_like(g)

    def run():
        if a.op == "wave":
            F.wave(prob, c, h, out_v, ws=ws)
        elif a.op == "wave_t":
            F.wave(prob, c, h, out_v, transpose=True, ws=ws)
        elif a.op == "forward":
            F.forward(prob, c, h, out_d, ws=ws)
        elif a.op == "adjoint":
            F.adjoint(prob, c, g, out_v, ws=ws)
        elif a.op == "project":
            F.project(prob, h, out_d)
        elif a.op == "backproject":
            F.backproject(prob, g, out_v)
        elif a.op == "ramp":
            F.ramp(prob, g, out_d)
        elif a.op == "fb":
            F.fb_solve(prob, c, g, 1e-3, 1e-3, 1, h=out_v.zero_(), ws=ws, history=False)

    run()
    torch.cuda.synchronize()
    F.profile_enable(True)
    F.profile_read()
    times = []
    for _ in range(a.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    prof = F.profile_read()
    F.profile_enable(False)
    res = {"op": a.op, "path": a.path, "n": n, "angles": a.angles, "nt": nt, "precision": a.precision,
           "ms": times, "ms_min": min(times)}
    if prof["step_launches"]:
        res["step_ms_avg"] = prof["step_ms"] / prof["step_launches"]
        res["step_gbs"] = prof["step_bytes"] / (prof["step_ms"] / 1e3) / 1e9
        res["voxel_steps_per_s"] = prof["steps"] * n**3 / (prof["step_ms"] / 1e3)
        res["step_ms_per_step"] = prof["step_ms"] / max(prof["steps"], 1)
    assert np.isfinite(out_v.double().sum().item()) or a.op in ("forward", "project", "ramp")
    print(json.dumps(res))


if __name__ == "__main__":
    main()
