"""GPU parity of the gradient regulariser R = 1/2 |grad h|^2 of the paper's
experiments (Sec. 5): its prox (I + a D^T D)^{-1} by DCT-II passes, and
Algorithms 8 and 9 with it, against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import (add_noise, axis, config, extend_speed, padded_axis,
                                           random_data, random_volume)

from tolerances import hist_dev, hist_tol, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [F.FP64, F.FP32, F.FP32_KAHAN]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build_lib.build()
    F.lib()


def dev(a, prob):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(F.torch_dtype(prob)).contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def as_input(a, prec):
    return a.astype(np.float32).astype(np.float64) if prec != F.FP64 else a


# 16: one tile; 37: ragged; 70: two row tiles and a ragged column tile
@pytest.mark.parametrize("prec", [F.FP64, F.FP32])
@pytest.mark.parametrize("n", [16, 37, 70])
def test_prox_grad(prec, n):
    f = as_input(random_volume(n, 300 + n), prec)
    prob = F.problem(n, 1.0, 4, prec)
    for a in (0.0, 0.7, 50.0):
        got = host(F.prox_grad(prob, dev(f, prob), a))
        assert rel(got, o.prox_grad(f, a)) < (1e-12 if prec == F.FP64 else 5e-6), a
    # in place
    t = dev(f, prob)
    F.prox_grad(prob, t, 3.0, out=t)
    assert rel(host(t), o.prox_grad(f, 3.0)) < (1e-12 if prec == F.FP64 else 5e-6)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("precond", [0, 1])
def test_fb_gradient_regulariser(prec, precond):
    n = 32 if precond == 0 else 20
    w = config(1, n=n)
    c, h = as_input(w.c, prec), as_input(w.h, prec)
    g = as_input(add_noise(o.forward(c, h, w.T, w.n_angles), random_data(w.n_angles, n, 3), 0.02),
                 prec)
    mask = np.broadcast_to((np.abs(axis(n)) > 0.25).astype(float), g.shape).copy()
    L = o.power(c, random_volume(n, 4), w.T, w.n_angles, precond=precond, iters=20, mask=mask)
    lam = 0.5 * L * (2.0 / n) ** 2  # a = s lambda / dx^2 = 0.5
    prob = F.problem(n, w.T, w.n_angles, prec, precond)
    h_gpu, st, hist = F.fb_solve_masked(prob, dev(c, prob), dev(g, prob), lam, 1.0 / L, 6,
                                        mask=dev(mask, prob), reg=F.REG_GRAD2)
    h_or, hist_or, k = o.fb_masked(c, g, w.T, lam, 1.0 / L, 6, mask=mask, precond=precond, reg=1)
    assert st["iters_done"] == k == 6
    assert rel(host(h_gpu), h_or) < tol(prec)
    for col in (0, 1, 3):
        assert hist_dev(hist, hist_or, cols=(col,)) < hist_tol(prec)


@pytest.mark.parametrize("prec", PRECS)
def test_two_step_gradient_regulariser_padded(prec):
    """Algorithm 9 as in the paper's experiments: padded wave grid, data for
    |xi| > a = 1 only (outside the source box), R = 1/2 |grad h|^2."""
    n, pad = 24, 8
    w = config(1, n=n, seed=23)
    c, h = as_input(extend_speed(w.c, pad), prec), as_input(w.h, prec)
    G = o.forward(c, h, w.T, w.n_angles, pad=pad)
    G = as_input(G * (np.abs(padded_axis(n, pad)) > 1.0), prec)
    prob = F.problem(n, w.T, w.n_angles, prec, pad=pad)
    h_gpu, st, hist = F.fb_two_step(prob, dev(c, prob), dev(G, prob), 0.5 * 0.3, 0.3, 5,
                                    reg=F.REG_GRAD2)
    h_or, hist_or, k = o.fb_two_step(c, G, w.T, 0.5 * 0.3, 0.3, 5, pad=pad, reg=1)
    assert st["iters_done"] == k == 5
    assert rel(host(h_gpu), h_or) < tol(prec)
    assert hist_dev(hist, hist_or, cols=(0,)) < hist_tol(prec)


def test_gradient_regulariser_rejects_support_and_unknown():
    w = config(1, n=16)
    prob = F.problem(16, w.T, 8)
    c = dev(w.c, prob)
    g = torch.zeros((8, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FFPATError):
        F.fb_solve_masked(prob, c, g, 0.1, 0.1, 1, support=dev(np.ones((16,) * 3), prob),
                          reg=F.REG_GRAD2)
    with pytest.raises(F.FFPATError):
        F.fb_solve_masked(prob, c, g, 0.1, 0.1, 1, reg=7)
