"""bench.py's JSON line (the keys the measurement contract asks for) on the
small 32^3 workload, and the FMA-rate probe the line uses for its
arithmetic-bound kernels."""
import json
import os
import subprocess
import sys

import pytest

from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fma_rate_probe():
    build_lib.build()
    fp64 = F.debug_fma_rate(F.FMA_FP64)
    fp32 = F.debug_fma_rate(F.FMA_FP32)
    fp32x2 = F.debug_fma_rate(F.FMA_FP32X2)
    assert 0 < fp64 < fp32 and fp32x2 > 0.5 * fp32
    assert fp32 < 2 * 152 * 128 * 2 * 2.1e9  # not above twice the clock-derived FP32 rate


def test_bench_line_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "cfg1",
                          "--steps", "3", "--warmup", "3", "--no-extras", "--ref-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "roofline",
              "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 3 and line["gpu_launches"] > 0
    assert line["config"]["workload"].startswith("small solve N=32^3")
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert 0 < r["frac"]
    e = line["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
