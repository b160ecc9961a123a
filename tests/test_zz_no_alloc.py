"""The allocation-free forward entry point (ffpat_forward_noalloc).

It serves callers that cannot allocate device memory or pass a workspace (code
inside an application that owns all device memory, or a real-time loop that
must never enter an allocator); its scratch is a static device array inside
the library.  This file is collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.  It passes alone
in a fresh process and after the other tests (the static scratch needs no
initial contents).
"""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import config, random_speed, random_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {F.FP64: 1e-10, F.FP32: 2e-5, F.FP32_KAHAN: 2e-5}


def _dev(a, prob):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(F.torch_dtype(prob))


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _as_input(a, prec):
    return a.astype(np.float32).astype(np.float64) if prec != F.FP64 else a


@pytest.mark.parametrize("prec", [F.FP64, F.FP32, F.FP32_KAHAN])
def test_noalloc_forward_matches_forward_and_oracle_twice(prec):
    """Two calls in a row on different inputs, each against ffpat_forward
    (same operator, workspace from torch) and against the FP64 oracle."""
    build_lib.build()
    w = config(1)  # N = 32, 24 angles, T = 1
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    inputs = [(w.c, w.h), (random_speed(w.n, 77), random_volume(w.n, 78))]
    for c, h in inputs:
        cd, hd = _dev(c, prob), _dev(h, prob)
        want = F.forward(prob, cd, hd)
        got = torch.full_like(want, float("nan"))
        F.forward_noalloc(prob, cd, hd, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        got = got.double().cpu().numpy()
        assert _rel(got, want.double().cpu().numpy()) < TOL[prec]
        g_or = o.forward(_as_input(c, prec), _as_input(h, prec), w.T, w.n_angles)
        assert _rel(got, g_or) < TOL[prec]


def test_noalloc_forward_allocates_nothing_after_the_first_call():
    """After a first call (which may load the library's device code and so
    commit the static array), further calls change neither the device's free
    memory nor torch's allocator."""
    build_lib.build()
    w = config(1)
    prob = F.problem(w.n, w.T, w.n_angles, F.FP32_KAHAN)
    cd, hd = _dev(w.c, prob), _dev(w.h, prob)
    g = torch.empty(F.data_shape(prob), dtype=torch.float32, device="cuda")
    F.forward_noalloc(prob, cd, hd, g)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(3):
        F.forward_noalloc(prob, cd, hd, g)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
    assert torch.isfinite(g).all()


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    build_lib.build()
    prob = F.problem(96, 0.5, 90, F.FP64)
    c = torch.ones((96, 96, 96), dtype=torch.float64, device="cuda")
    g = torch.empty((90, 96, 96), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FFPATError) as e:
        F.forward_noalloc(prob, c, c, g)
    assert e.value.code == F.EINVAL and "static scratch" in str(e.value)
    # the bound is on the wave grid: a padded N = 64 problem is too large
    padded = F.problem(64, 0.2, 180, F.FP64, pad=8)
    cw = torch.ones((80, 80, 80), dtype=torch.float64, device="cuda")
    h64 = torch.ones((64, 64, 64), dtype=torch.float64, device="cuda")
    gw = torch.empty((180, 80, 80), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FFPATError) as e:
        F.forward_noalloc(padded, cw, h64, gw)
    assert e.value.code == F.EINVAL and "static scratch" in str(e.value)
    # the largest advertised size is accepted
    big = F.problem(64, 0.2, 180, F.FP64)
    c64 = torch.ones((64, 64, 64), dtype=torch.float64, device="cuda")
    g64 = torch.empty((180, 64, 64), dtype=torch.float64, device="cuda")
    F.forward_noalloc(big, c64, c64, g64)
    torch.cuda.synchronize()
    assert torch.isfinite(g64).all()
