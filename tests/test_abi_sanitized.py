"""Host-side code of the library under AddressSanitizer and
UndefinedBehaviorSanitizer (CPU only, no GPU): the sanitizer build of
libffpat (device code unchanged) is loaded into a child process that preloads
the sanitizer runtimes, and every host-only path is exercised: argument
validation, workspace carve sizes (padded problems included), time-step
rules, angle tables, checkpoint sizes, error paths of the compute entry
points and of the server.  Any sanitizer report fails the test."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

from paper_1901_06503_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1901_06503_gb300 import ffpat as F
L = F.lib()
for name in F.header_symbols():
    getattr(L, name)
assert L.ffpat_version().startswith(b"ffpat")
sizes = []
for n, pad, prec, nth in [(16, 0, 0, 8), (33, 0, 2, 5), (32, 8, 1, 24), (64, 64, 2, 180),
                          (0, 0, 0, 8), (5000, 0, 0, 8), (16, -1, 0, 8), (2048, 1025, 0, 8),
                          (16, 0, 7, 8), (16, 0, 0, 0)]:
    p = F.problem(n, 1.0, nth, prec, pad=pad)
    sizes.append(L.ffpat_workspace_bytes(ctypes.byref(p)))
    L.ffpat_last_error()
assert sizes[0] > 0 and sizes[4] == 0 and sizes[5] == 0 and sizes[6] == 0
p = F.problem(64, 1.2, 90, F.FP32_KAHAN, pad=16)
nt, dt, ns = F.problem_info(p, 1.3)
assert nt > 0 and ns > 0
cs = np.zeros(2 * 90)
assert L.ffpat_debug_tables(ctypes.byref(p), cs.ctypes.data_as(ctypes.c_void_p)) == 0
assert L.ffpat_ckpt_bytes(ctypes.byref(F.problem(64, 1.0, 8)), 100, 16) > 0
assert L.ffpat_ckpt_bytes(ctypes.byref(p), 100, 16) == 0
assert L.ffpat_forward(ctypes.byref(p), None, None, None, None, 0, None) == F.EINVAL
fake = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
assert L.ffpat_fb_solve(ctypes.byref(p), None, None, 0.0, 1.0, 1, 0.0, None, None, None,
                        fake, 1024, None) == F.ENOMEM
assert L.ffpat_set_stencil_path(7) == F.EINVAL
assert L.ffpat_debug_wait_timeout(0, None) == F.EINVAL
srv = ctypes.c_void_p()
rc = L.ffpat_server_create(ctypes.c_size_t(1 << 30), 4, ctypes.byref(srv))
if rc == 0:
    assert L.ffpat_server_destroy(srv) == 0
print("sanitized host paths ok")
'''


def _runtime(name):
    cc = shutil.which("gcc")
    if not cc:
        return None
    path = subprocess.run([cc, f"-print-file-name={name}"], capture_output=True,
                          text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_host_paths_under_asan_ubsan():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("sanitizer runtimes not installed")
    try:
        lib = build_lib.build_sanitized()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e)[:200])
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", FFPAT_LIB=lib,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + PROBE], env=env,
                       capture_output=True, text=True, timeout=300)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-3000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-3000:]
    assert "sanitized host paths ok" in out
