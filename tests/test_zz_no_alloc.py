"""The allocation-free forward entry point (ffpat_forward_noalloc).

It serves callers that cannot allocate device memory or pass a workspace; its
scratch is a static device array inside the library.  This file is collected
last on purpose: if it fails, a run that stops at the first failure has
already run every other test.  It passes alone in a fresh process and after
the other tests (the static scratch needs no initial contents).
"""
import ctypes

import numpy as np
import pytest

from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import config, random_speed, random_volume

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {F.FP64: 1e-10, F.FP32: 2e-5, F.FP32_KAHAN: 2e-5}


def _dev(a, prob):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(F.torch_dtype(prob))


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


@pytest.mark.parametrize("prec", [F.FP64, F.FP32, F.FP32_KAHAN])
def test_noalloc_forward_matches_forward_twice(prec):
    build_lib.build()
    w = config(1)  # N = 32, 24 angles, T = 1
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    inputs = [(w.c, w.h), (random_speed(w.n, 77), random_volume(w.n, 78))]
    for c, h in inputs:  # two calls in a row, different inputs
        cd, hd = _dev(c, prob), _dev(h, prob)
        want = F.forward(prob, cd, hd)
        got = torch.full_like(want, float("nan"))
        F.forward_noalloc(prob, cd, hd, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, want) < TOL[prec]


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    build_lib.build()
    prob = F.problem(96, 0.5, 90, F.FP64)
    c = torch.ones((96, 96, 96), dtype=torch.float64, device="cuda")
    g = torch.empty((90, 96, 96), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FFPATError) as e:
        F.forward_noalloc(prob, c, c, g)
    assert e.value.code == F.EINVAL and "static scratch" in str(e.value)
    # the largest advertised size is accepted
    big = F.problem(64, 0.2, 180, F.FP64)
    c64 = torch.ones((64, 64, 64), dtype=torch.float64, device="cuda")
    g64 = torch.empty((180, 64, 64), dtype=torch.float64, device="cuda")
    F.forward_noalloc(big, c64, c64, g64)
    torch.cuda.synchronize()
    assert torch.isfinite(g64).all()
