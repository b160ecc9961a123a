"""GPU parity on the padded wave grid (V_T of the wave model, the enlarged
computational domain of the paper's experiments, Sec. 5): the wave runs on
Nw = N + 2 pad points per axis, sources and images stay on the N^3 box, and
the data are the projections of the whole wave grid (n_angles x Nw x Nw).
Each case is compared with the oracle's padded operators element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import (add_noise, config, extend_speed, padded_axis,
                                           random_data, random_volume)

from tolerances import hist_dev, hist_tol, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {F.FP64: 1e-10, F.FP32: 2e-5, F.FP32_KAHAN: 2e-5}
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


def case(n, pad, prec, seed=1):
    """Config-1 sources and speed on an n^3 box, the speed continued outwards."""
    w = config(1, n=n, seed=seed)
    return w, as_input(extend_speed(w.c, pad), prec), as_input(w.h, prec)


# (32, 8): wave grid 48^3, TMA-aligned; (20, 3): 26^3, the plain stencil for FP32
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,pad", [(32, 8), (20, 3)])
def test_padded_forward_adjoint(prec, n, pad):
    w, c, h = case(n, pad, prec)
    prob = F.problem(n, w.T, w.n_angles, prec, pad=pad)
    g_gpu = host(F.forward(prob, dev(c, prob), dev(h, prob)))
    g_or = o.forward(c, h, w.T, w.n_angles, pad=pad)
    assert rel(g_gpu, g_or) < TOL[prec]
    gd = as_input(add_noise(g_or, random_data(w.n_angles, n + 2 * pad, 7), 0.01), prec)
    a_gpu = host(F.adjoint(prob, dev(c, prob), dev(gd, prob)))
    assert rel(a_gpu, o.adjoint(c, gd, w.T, pad=pad)) < TOL[prec]
    # the padding matters here: the box-sized operator differs on the box's rays
    box = g_or[:, pad:-pad, pad:-pad]
    assert rel(box, o.forward(w.c, w.h, w.T, w.n_angles)) > 100 * TOL[prec]


@pytest.mark.parametrize("n,pad", [(32, 8), (20, 3)])
def test_padded_projection_fp64_bit_exact(n, pad):
    """P of the wave grid in FP64 reproduces the oracle bit for bit (same
    sample arithmetic with L = Nw / N), and the sample tables agree."""
    nw, nth = n + 2 * pad, 7
    p = random_volume(nw, 9)
    prob = F.problem(n, 1.0, nth, pad=pad)
    g = host(F.project(prob, dev(p, prob)))
    assert np.array_equal(g, o.project(p, nth, nimg=n))
    rng = np.random.default_rng(10)
    ns = 2 * int(np.ceil(nw / np.sqrt(2.0)))
    jkm = np.stack([rng.integers(0, nth, 500), rng.integers(0, nw, 500),
                    rng.integers(0, ns, 500)], axis=1)
    ij, f = F.debug_samples(prob, jkm)
    ij_or, f_or = o.sample_points(nw, nth, jkm, nimg=n)
    assert np.array_equal(ij, ij_or) and np.array_equal(f, f_or)
    h = host(F.backproject(prob, dev(g, prob)))
    assert rel(h, o.backproject(g, nw, nimg=n)) < 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_padded_wave_and_transpose(prec):
    n, pad, T = 24, 6, 0.8
    w, c, _ = case(n, pad, prec, seed=11)
    x = as_input(random_volume(n, 12), prec)
    prob = F.problem(n, T, 4, prec, pad=pad)
    assert rel(host(F.wave(prob, dev(c, prob), dev(x, prob))), o.wave_pad(c, x, T, pad)) < TOL[prec]
    u = as_input(random_volume(n + 2 * pad, 13), prec)
    wt = host(F.wave(prob, dev(c, prob), dev(u, prob), transpose=True))
    assert rel(wt, o.wave_pad(c, u, T, pad, transpose=True)) < TOL[prec]


def test_padded_opnorm_fp64():
    n, pad = 16, 4
    w, c, _ = case(n, pad, F.FP64, seed=13)
    v0 = random_volume(n, 14)
    prob = F.problem(n, w.T, 8, pad=pad)
    got = F.opnorm(prob, dev(c, prob), dev(v0, prob), iters=20)
    assert abs(got - o.power(c, v0, w.T, 8, iters=20, pad=pad)) < 1e-10 * got


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("precond", [0, 1])
def test_padded_limited_view_fb(prec, precond):
    """The paper's experimental setting: padded wave grid, data only for
    |xi| > a = 1 (chi_M: the rays that miss the source box) and a source
    support chi_V inside the box."""
    n, pad = 24, 8
    w, c, h = case(n, pad, prec, seed=15)
    g = as_input(add_noise(o.forward(c, h, w.T, w.n_angles, pad=pad),
                           random_data(w.n_angles, n + 2 * pad, 16), 0.01), prec)
    mask = np.broadcast_to((np.abs(padded_axis(n, pad)) > 1.0).astype(float), g.shape).copy()
    sup = np.zeros((n, n, n))
    sup[2:-2, 2:-2, 2:-2] = 1.0
    L = o.power(c, random_volume(n, 17), w.T, w.n_angles, precond=precond, iters=20, pad=pad,
                mask=mask)
    prob = F.problem(n, w.T, w.n_angles, prec, precond, pad=pad)
    h_gpu, st, hist = F.fb_solve_masked(prob, dev(c, prob), dev(g, prob), w.lam, 1.0 / L, 6,
                                        mask=dev(mask, prob), support=dev(sup, prob))
    h_or, hist_or, k = o.fb_masked(c, g, w.T, w.lam, 1.0 / L, 6, mask=mask, support=sup,
                                   precond=precond, pad=pad)
    hg = host(h_gpu)
    assert st["iters_done"] == k == 6
    assert np.all(hg[sup == 0] == 0)
    assert rel(hg, h_or) < tol(prec)
    for col in (0, 1, 3):
        assert hist_dev(hist, hist_or, cols=(col,)) < hist_tol(prec)


@pytest.mark.parametrize("prec", PRECS)
def test_padded_two_step(prec):
    n, pad = 24, 8
    w, c, h = case(n, pad, prec, seed=19)
    G = as_input(o.forward(c, h, w.T, w.n_angles, pad=pad), prec)
    prob = F.problem(n, w.T, w.n_angles, prec, pad=pad)
    h_gpu, st, hist = F.fb_two_step(prob, dev(c, prob), dev(G, prob), w.lam, 0.5, 5)
    h_or, hist_or, k = o.fb_two_step(c, G, w.T, w.lam, 0.5, 5, pad=pad)
    assert st["iters_done"] == k == 5
    assert rel(host(h_gpu), h_or) < tol(prec)


def test_padding_rejected_by_gradient_path():
    n, pad = 16, 4
    w, c, h = case(n, pad, F.FP32, seed=21)
    prob = F.problem(n, w.T, 8, F.FP32, pad=pad)
    with pytest.raises(F.FFPATError):
        F.forward_ckpt(prob, dev(c, prob), dev(h, prob), 4,
                       torch.zeros(1 << 20, dtype=torch.uint8, device="cuda"))
