"""GPU parity: every hot-path step of the CUDA library against the FP64 oracle
on the same seeded inputs.

Tolerances (relative L2): 1e-10 for FP64 problems, 2e-5 for the FP32 and
FP32-Kahan wavefields; bit-exact for the FP64 projection's index arithmetic and
for the FP64 projection itself on identical input.
"""
import os

import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import (add_noise, config, random_data, random_speed,
                                           random_volume)
from tolerances import FP32_TOL, hist_dev, hist_tol, tol

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
    """What the GPU receives, in float64 (FP32 problems get rounded inputs)."""
    return a.astype(np.float32).astype(np.float64) if prec != F.FP64 else a


# ---------------------------------------------------------- index tables --

def test_sample_index_arithmetic_bit_exact():
    rng = np.random.default_rng(5)
    for n, nth in [(32, 24), (33, 7), (128, 90), (384, 180)]:
        ns = o.ray_samples(n)
        jkm = np.stack([rng.integers(0, nth, 4000), rng.integers(0, n, 4000),
                        rng.integers(0, ns, 4000)], axis=1).astype(np.int32)
        prob = F.problem(n, 1.0, nth)
        ij_g, f_g = F.debug_samples(prob, jkm)
        ij_o, f_o = o.sample_points(n, nth, jkm)
        assert np.array_equal(ij_g, ij_o)
        assert np.array_equal(f_g, f_o)


# ----------------------------------------------------------- projection --

@pytest.mark.parametrize("n,nth", [(24, 6), (33, 7), (40, 13)])
def test_project_fp64_bit_exact(n, nth):
    p = random_volume(n, 100 + n)
    prob = F.problem(n, 1.0, nth)
    g = host(F.project(prob, dev(p, prob)))
    assert np.array_equal(g, o.project(p, nth))


# planes too large for shared memory: FP64 (from N ~ 155) from global memory,
# steep angles through a transposed copy; FP32 (from N ~ 220) band by band,
# bands visited in each ray's order (odd angle counts put angles on both sides
# of 90 degrees in one call)
@pytest.mark.parametrize("n,pad,nth", [(160, 0, 8), (120, 20, 7), (256, 0, 5)])
def test_project_fp64_large_planes_bit_exact(n, pad, nth):
    nw = n + 2 * pad
    p = random_volume(nw, 110 + n)
    prob = F.problem(n, 1.0, nth, pad=pad)
    g = host(F.project(prob, dev(p, prob)))
    assert np.array_equal(g, o.project(p, nth, nimg=n))


@pytest.mark.parametrize("n,pad,nth", [(232, 0, 6), (200, 28, 7)])
def test_project_fp32_large_planes(n, pad, nth):
    p = random_volume(n + 2 * pad, 120)
    prob = F.problem(n, 1.0, nth, F.FP32, pad=pad)
    g = host(F.project(prob, dev(p, prob)))
    assert rel(g, o.project(as_input(p, F.FP32), nth, nimg=n)) < 5e-7


def test_project_fp32_global_fallback(tmp_path):
    """The FP32 global-memory projection (planes too large even for a band,
    N >= 1024), forced at N = 232 with FFPAT_PROJECT_BAND=0 in a child
    process, steep angles through the transposed copy."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n, nth = 232, 8
    p = random_volume(n, 130).astype(np.float32)
    np.save(tmp_path / "p.npy", p)
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_1901_06503_gb300 import ffpat as F\n"
        f"p = np.load({str(tmp_path / 'p.npy')!r})\n"
        f"prob = F.problem({n}, 1.0, {nth}, F.FP32)\n"
        "g = F.project(prob, torch.as_tensor(p, device='cuda'))\n"
        "torch.cuda.synchronize()\n"
        f"np.save({str(tmp_path / 'g.npy')!r}, g.cpu().numpy())\n")
    env = dict(os.environ, FFPAT_PROJECT_BAND="0")
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=300)
    g = np.load(tmp_path / "g.npy").astype(np.float64)
    assert rel(g, o.project(p.astype(np.float64), nth)) < 5e-7


# FP32 with even N and an even angle count 2h evaluates each bilinear sample
# of theta's lattice once for the four angles theta, theta + 90, 180 - theta,
# 90 - theta (k_project_quad); odd cases take the one-angle kernels.  The
# cases span several 32 x 16 lattice tiles with ragged edges, h odd and even
# (the 45-degree class), the pair 0 / 90 alone, one band (up to N = 192) and
# band by band (the N = 232 case of the large planes)
PROJ_CASES = [(24, 6), (33, 7), (40, 12), (64, 90), (24, 4), (48, 16), (16, 2), (100, 10),
              (130, 14), (40, 13), (192, 12)]


def _check_angles(g, want, tol=1e-6):
    assert rel(g, want) < 5e-7
    for a in range(want.shape[0]):  # every angle: each class writes four of them
        assert rel(g[a], want[a]) < tol, a


@pytest.mark.parametrize("prec", [F.FP32])
@pytest.mark.parametrize("n,nth", PROJ_CASES)
def test_project_fp32(n, nth, prec):
    p = random_volume(n, 200 + n)
    prob = F.problem(n, 1.0, nth, prec)
    g = host(F.project(prob, dev(p, prob)))
    _check_angles(g, o.project(as_input(p, prec), nth))


def _project_child(tmp_path, cases, env_key, env_val, seed0):
    """Run F.project in a child process with one environment knob set."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for i, (n, nth) in enumerate(cases):
        np.save(tmp_path / f"p{i}.npy", random_volume(n, seed0 + n).astype(np.float32))
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_1901_06503_gb300 import ffpat as F\n"
        f"for i, (n, nth) in enumerate({cases!r}):\n"
        f"    p = np.load({str(tmp_path)!r} + f'/p{{i}}.npy')\n"
        "    prob = F.problem(n, 1.0, nth, F.FP32)\n"
        "    g = F.project(prob, torch.as_tensor(p, device='cuda'))\n"
        "    torch.cuda.synchronize()\n"
        f"    np.save({str(tmp_path)!r} + f'/g{{i}}.npy', g.cpu().numpy())\n")
    env = dict(os.environ, **{env_key: env_val})
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=300)
    out = []
    for i, (n, nth) in enumerate(cases):
        p = np.load(tmp_path / f"p{i}.npy").astype(np.float64)
        g = np.load(tmp_path / f"g{i}.npy").astype(np.float64)
        out.append((p, g))
    return out


def test_project_fp32_one_angle_kernels(tmp_path):
    """The one-angle FP32 projections on cases the four-angle kernel takes by
    default (whole plane in shared memory; band by band at N = 232), forced
    with FFPAT_PROJECT_QUAD=0 in a child process."""
    cases = [(24, 6), (64, 90), (192, 12), (232, 6)]
    for (n, nth), (p, g) in zip(cases, _project_child(tmp_path, cases, "FFPAT_PROJECT_QUAD", "0",
                                                       210)):
        assert rel(g, o.project(p, nth)) < 5e-7, (n, nth)


def test_project_fp32_deterministic():
    """The four-angle projection sums in a fixed order: two calls agree bit
    for bit (whole plane, and band by band at N = 232)."""
    for n, nth in ((64, 90), (192, 12), (232, 6)):
        p = random_volume(n, 220 + n)
        prob = F.problem(n, 1.0, nth, F.FP32)
        pd = dev(p, prob)
        g1 = host(F.project(prob, pd))
        g2 = host(F.project(prob, pd))
        assert np.array_equal(g1, g2)


# FP32 with even N and an even angle count 2h applies each weight set to the
# four angles theta, theta + 90, 180 - theta, 90 - theta ((24, 6) and (64, 90):
# h odd; (40, 12), (24, 4), (48, 16): h even, with the 45-degree class; (16, 2):
# the pair 0, 90 alone); the others take the per-angle gather
BP_CASES = [(24, 6), (33, 7), (40, 13), (40, 12), (33, 8), (64, 90), (24, 4), (48, 16), (16, 2)]


@pytest.mark.parametrize("prec", [F.FP64, F.FP32])
@pytest.mark.parametrize("n,nth", BP_CASES)
def test_backproject(n, nth, prec):
    g = random_data(nth, n, 300 + n)
    prob = F.problem(n, 1.0, nth, prec)
    h = host(F.backproject(prob, dev(g, prob)))
    want = o.backproject(as_input(g, prec), n)
    assert rel(h, want) < (1e-12 if prec == F.FP64 else 5e-7)


@pytest.mark.parametrize("knob", ["FFPAT_BACKPROJECT_QUAD", "FFPAT_BACKPROJECT_PAIR"])
def test_backproject_fp32_other_kernels(tmp_path, knob):
    """The FP32 transposes the four-angle kernel replaces, forced in a child
    process: the theta / theta + 90 pair (QUAD=0) and the per-angle gather
    (PAIR=0), on the even cases."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cases = [(24, 6), (40, 12), (64, 90)]
    for i, (n, nth) in enumerate(cases):
        np.save(tmp_path / f"g{i}.npy", random_data(nth, n, 300 + n).astype(np.float32))
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_1901_06503_gb300 import ffpat as F\n"
        f"for i, (n, nth) in enumerate({cases!r}):\n"
        f"    g = np.load({str(tmp_path)!r} + f'/g{{i}}.npy')\n"
        "    prob = F.problem(n, 1.0, nth, F.FP32)\n"
        "    h = F.backproject(prob, torch.as_tensor(g, device='cuda'))\n"
        "    torch.cuda.synchronize()\n"
        f"    np.save({str(tmp_path)!r} + f'/h{{i}}.npy', h.cpu().numpy())\n")
    env = dict(os.environ, **{knob: "0"})
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=300)
    for i, (n, nth) in enumerate(cases):
        g = np.load(tmp_path / f"g{i}.npy").astype(np.float64)
        h = np.load(tmp_path / f"h{i}.npy").astype(np.float64)
        assert rel(h, o.backproject(g, n)) < 5e-7, (knob, n, nth)


# (96, 20): 1920 rows, more than the grid's 1216 CTAs, so CTAs walk several rows
@pytest.mark.parametrize("prec", [F.FP64, F.FP32])
@pytest.mark.parametrize("n,nth", [(24, 6), (33, 3), (130, 2), (96, 20)])
def test_ramp(n, nth, prec):
    r = random_data(nth, n, 400 + n)
    prob = F.problem(n, 1.0, nth, prec)
    out = host(F.ramp(prob, dev(r, prob)))
    assert rel(out, o.ramp(as_input(r, prec))) < (1e-12 if prec == F.FP64 else 2e-6)


# ----------------------------------------------------------- wave operator --

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,T", [(24, 0.6), (33, 0.45), (40, 0.02)])
def test_wave_and_transpose(n, T, prec):
    c = as_input(random_speed(n, 500 + n), prec)
    h = as_input(random_volume(n, 501 + n), prec)
    prob = F.problem(n, T, 4, prec)
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    kap = o.kappa(n, dt, c)
    w = host(F.wave(prob, dev(c, prob), dev(h, prob)))
    assert rel(w, o.wave(kap, h, nt)) < TOL[prec]
    wt = host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True))
    assert rel(wt, o.wave_adjoint(kap, h, nt)) < TOL[prec]


# ----------------------------------------------------- composite operator --

@pytest.mark.parametrize("prec", PRECS)
def test_forward_adjoint_config1(prec):
    w = config(1)
    c, h = as_input(w.c, prec), as_input(w.h, prec)
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    g_gpu = host(F.forward(prob, dev(c, prob), dev(h, prob)))
    g_or = o.forward(c, h, w.T, w.n_angles)
    assert rel(g_gpu, g_or) < TOL[prec]
    gd = as_input(add_noise(g_or, w.noise, w.noise_rel), prec)
    a_gpu = host(F.adjoint(prob, dev(c, prob), dev(gd, prob)))
    assert rel(a_gpu, o.adjoint(c, gd, w.T)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_forward_adjoint_ragged(prec):
    n, nth, T = 37, 11, 0.5
    c = as_input(random_speed(n, 601), prec)
    h = as_input(random_volume(n, 602), prec)
    g = as_input(random_data(nth, n, 603), prec)
    prob = F.problem(n, T, nth, prec)
    assert rel(host(F.forward(prob, dev(c, prob), dev(h, prob))), o.forward(c, h, T, nth)) < TOL[prec]
    assert rel(host(F.adjoint(prob, dev(c, prob), dev(g, prob))), o.adjoint(c, g, T)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nth", [(1, 1), (2, 1), (3, 2), (4, 1), (8, 1)])
def test_degenerate_grids(prec, n, nth):
    """The smallest grids and a single angle: one to three cells per axis
    (the plain kernels, N_s = 2 samples per ray), 4^3 and 8^3 (the TMA and
    resident paths) with one angle; forward and adjoint against the oracle."""
    T = 0.3
    c = as_input(random_speed(n, 650 + n), prec)
    h = as_input(random_volume(n, 651 + n), prec)
    g = as_input(random_data(nth, n, 652 + n), prec)
    prob = F.problem(n, T, nth, prec)
    assert rel(host(F.forward(prob, dev(c, prob), dev(h, prob))), o.forward(c, h, T, nth)) < TOL[prec]
    assert rel(host(F.adjoint(prob, dev(c, prob), dev(g, prob))), o.adjoint(c, g, T)) < TOL[prec]
    assert F.device_status() == 0


def test_dot_product_gpu_fp64():
    n, nth, T = 36, 9, 0.7
    prob = F.problem(n, T, nth)
    c = dev(random_speed(n, 701), prob)
    h = dev(random_volume(n, 702), prob)
    g = dev(random_data(nth, n, 703), prob)
    Ah = F.forward(prob, c, h)
    Atg = F.adjoint(prob, c, g)
    lhs = float((Ah * g).sum())
    rhs = float((h * Atg).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(Ah.norm() * g.norm())


@pytest.mark.parametrize("prec", PRECS)
def test_forward_adjoint_config2_full(prec):
    """N = 128, 90 angles, T = 1.2 (333 steps): the whole operator pair."""
    w = config(2)
    c, h = as_input(w.c, prec), as_input(w.h, prec)
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    g_or = o.forward(c, h, w.T, w.n_angles)
    g_gpu = host(F.forward(prob, dev(c, prob), dev(h, prob)))
    assert rel(g_gpu, g_or) < TOL[prec]
    gd = as_input(add_noise(g_or, w.noise, w.noise_rel), prec)
    a_gpu = host(F.adjoint(prob, dev(c, prob), dev(gd, prob)))
    assert rel(a_gpu, o.adjoint(c, gd, w.T)) < TOL[prec]


def test_config2_fp32_vs_fp64_100_iterations():
    """The 128^3 solve (90 angles, T = 1.2, 2 % noise, identity Lambda) for
    the workload's 100 FB iterations in FP32 and FP32-Kahan against the FP64
    GPU path with the same step (1/L from 8 oracle power iterations), and the
    FP64 GPU path against the oracle over the first 10 iterations (the
    oracle's scope at this size)."""
    w = config(2)
    c64 = w.c
    g64 = add_noise(o.forward(c64, w.h, w.T, w.n_angles), w.noise, w.noise_rel)
    s = 1.0 / o.power(c64, np.ones_like(c64), w.T, w.n_angles, iters=8)
    res = {}
    for prec in PRECS:
        prob = F.problem(w.n, w.T, w.n_angles, prec)
        h, st, _ = F.fb_solve(prob, dev(c64, prob), dev(g64, prob), w.lam, s, 100,
                              history=False)
        assert st["iters_done"] == 100
        res[prec] = host(h)
    for prec in (F.FP32, F.FP32_KAHAN):
        assert rel(res[prec], res[F.FP64]) < FP32_TOL
    p64 = F.problem(w.n, w.T, w.n_angles, F.FP64)
    h10, _, _ = F.fb_solve(p64, dev(c64, p64), dev(g64, p64), w.lam, s, 10, history=False)
    h_or, _, k = o.fb(c64, g64, w.T, w.lam, s, 10)
    assert k == 10
    assert rel(host(h10), h_or) < tol(F.FP64)


# ------------------------------------------------------------ Algorithm 8 --

def fb_case(prec, precond=0, n=None):
    w = config(1, n=n)
    c, htrue = as_input(w.c, prec), w.h
    g = add_noise(o.forward(c, htrue, w.T, w.n_angles), w.noise, w.noise_rel)
    g = as_input(g, prec)
    L = o.power(c, random_volume(w.n, 9), w.T, w.n_angles, precond=precond, iters=20)
    return w, c, g, 1.0 / L


@pytest.mark.parametrize("prec", PRECS)
def test_fb_config1(prec):
    w, c, g, s = fb_case(prec)
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    h_gpu, st, hist = F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, s, w.iters)
    h_or, hist_or, k = o.fb(c, g, w.T, w.lam, s, w.iters)
    assert st["iters_done"] == k == w.iters
    assert rel(host(h_gpu), h_or) < tol(prec)
    assert hist_dev(hist, hist_or) < hist_tol(prec)
    assert abs(st["objective"] - hist_or[-1, 0]) < hist_tol(prec) * abs(hist_or[-1, 0])


def test_fb_preconditioned_fp64():
    w, c, g, s = fb_case(F.FP64, precond=1, n=20)
    prob = F.problem(w.n, w.T, w.n_angles, F.FP64, precond=1)
    h_gpu, st, hist = F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, s, 6)
    h_or, hist_or, k = o.fb(c, g, w.T, w.lam, s, 6, precond=1)
    assert rel(host(h_gpu), h_or) < 1e-10
    assert np.max(np.abs(hist[:, 0] - hist_or[:, 0]) / np.abs(hist_or[:, 0])) < 1e-9


def test_fb_deterministic_fp64():
    w, c, g, s = fb_case(F.FP64)
    prob = F.problem(w.n, w.T, w.n_angles)
    outs = [host(F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, s, 3)[0]) for _ in range(2)]
    assert np.array_equal(outs[0], outs[1])


def test_fb_tolerance_and_warm_start():
    w, c, g, s = fb_case(F.FP64)
    prob = F.problem(w.n, w.T, w.n_angles)
    h0 = np.maximum(w.h + 0.05 * random_volume(w.n, 33), 0)
    h_gpu, st, hist = F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, s, 50, h=dev(h0, prob),
                                 tol=2e-2)
    h_or, hist_or, k = o.fb(c, g, w.T, w.lam, s, 50, h0=h0, tol=2e-2)
    assert st["iters_done"] == k < 50
    assert rel(host(h_gpu), h_or) < 1e-10


@pytest.mark.parametrize("precond", [0, 1])
def test_opnorm_fp64(precond):
    n, nth, T = 20, 8, 0.6
    c = random_speed(n, 801)
    v0 = random_volume(n, 802)
    prob = F.problem(n, T, nth, F.FP64, precond)
    est = F.opnorm(prob, dev(c, prob), dev(v0, prob), iters=20)
    want = o.power(c, v0, T, nth, precond=precond, iters=20)
    assert abs(est - want) < 1e-10 * want


def test_fb_automatic_step():
    w, c, g, s = fb_case(F.FP64)
    prob = F.problem(w.n, w.T, w.n_angles)
    _, st, _ = F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, 0.0, 1)
    assert abs(st["step"] - s) < 0.05 * s and st["opnorm_sq"] > 0


# --------------------------------------------------------------- errors --

def test_rejects_nonpositive_speed():
    n = 16
    prob = F.problem(n, 0.5, 4)
    c = random_speed(n, 1)
    c[3, 4, 5] = 0.0
    with pytest.raises(F.FFPATError) as e:
        F.forward(prob, dev(c, prob), dev(random_volume(n, 2), prob))
    assert e.value.code == F.EINVAL


# ------------------------------------------- full sizes, bench launch shape --

def test_full_size_n384_fp32_spot_checks():
    """N = 384, 180 angles (the large solve): the stencil launch and the
    projection in the bench's launch configuration, checked where the oracle
    can follow -- one time step on the whole grid and a sample of rays --
    and the transpose pair through the dot product."""
    n, nth = 384, 180
    rng = np.random.default_rng(11)
    c = as_input(np.clip(1 + 0.2 * rng.standard_normal((n, n, n)), 0.75, 1.4), F.FP32)
    h = as_input(rng.standard_normal((n, n, n)), F.FP32)
    cmax = c.max()
    T1 = 0.3 * (2.0 / n) / cmax * 0.999  # exactly one time step
    for prec in (F.FP32, F.FP32_KAHAN):
        prob = F.problem(n, T1, nth, prec)
        nt, dt = o.time_steps(n, T1, 0.3, cmax)
        assert nt == 1
        w1 = host(F.wave(prob, dev(c, prob), dev(h, prob)))
        assert rel(w1, o.wave(o.kappa(n, dt, c), h, 1)) < 1e-6
    prob = F.problem(n, 1.0, nth, F.FP32)
    g = host(F.project(prob, dev(h, prob)))
    jlk = np.stack([rng.integers(0, nth, 3000), rng.integers(0, n, 3000),
                    rng.integers(0, n, 3000)], axis=1)
    want = o.project_rays(h, nth, jlk)
    got = g[jlk[:, 0], jlk[:, 1], jlk[:, 2]]
    assert rel(got, want) < 1e-6
    gt = dev(random_data(nth, n, 12), prob)
    bp = F.backproject(prob, gt)
    hd = dev(h, prob)
    lhs = float((F.project(prob, hd).double() * gt.double()).sum())
    rhs = float((hd.double() * bp.double()).sum())
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_full_size_n384_two_step_pass():
    """N = 384 FP32-Kahan as the large solve runs it: the start step, then
    one two-step pass (the automatic choice at this size), bit for bit the
    step-by-step loop and within tolerance of the oracle, for W and W^T."""
    n = 384
    rng = np.random.default_rng(13)
    c = as_input(np.clip(1 + 0.2 * rng.standard_normal((n, n, n)), 0.75, 1.4), F.FP32)
    h = as_input(rng.standard_normal((n, n, n)), F.FP32)
    cmax = c.max()
    T3 = 3 * 0.3 * (2.0 / n) / cmax * 0.999  # exactly three time steps
    nt, dt = o.time_steps(n, T3, 0.3, cmax)
    assert nt == 3
    prob = F.problem(n, T3, 4, F.FP32_KAHAN)
    outs = {}
    try:
        for path in (0, 2):
            F.set_stencil_path(path)
            outs[path] = (host(F.wave(prob, dev(c, prob), dev(h, prob))),
                          host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True)))
    finally:
        F.set_stencil_path(0)
    assert np.array_equal(outs[0][0], outs[2][0]) and np.array_equal(outs[0][1], outs[2][1])
    kap = o.kappa(n, dt, c)
    assert rel(outs[0][0], o.wave(kap, h, nt)) < 1e-6
    assert rel(outs[0][1], o.wave_adjoint(kap, h, nt)) < 1e-6
    assert F.device_status() == 0


def _config5_problem():
    w = config(5)
    prec = F.FP32_KAHAN
    c, h = as_input(w.c, prec), as_input(w.h, prec)
    return w, prec, c, h, F.problem(w.n, w.T, w.n_angles, prec, w.precond)


def test_config5_forward_adjoint_full_length():
    """The large solve's operator pair at full length: N = 384, 180 angles,
    T = 1.5 (1344 leapfrog steps: the start step, then two steps per pass,
    the automatic path at this size), FP32-Kahan.  The forward of the
    workload's phantom and the adjoint of its noisy data (Problem 1 of
    Sec. 2.1), element by element against the oracle on every projection and
    on the whole grid."""
    w, prec, c, h, prob = _config5_problem()
    cd = dev(c, prob)
    F.profile_enable(True)
    F.profile_read()
    g_gpu = host(F.forward(prob, cd, dev(h, prob)))
    prof = F.profile_read()
    F.profile_enable(False)
    nt, _ = o.time_steps(w.n, w.T, 0.3, float(c.max()))
    assert nt == 1344 and prof["steps"] == nt
    assert prof["step_launches"] < 0.51 * nt  # two steps per pass
    g_or = o.forward(c, h, w.T, w.n_angles)
    assert rel(g_gpu, g_or) < FP32_TOL
    gd = as_input(add_noise(g_or, w.noise, w.noise_rel), prec)
    del g_gpu, g_or
    a_gpu = host(F.adjoint(prob, cd, dev(gd, prob)))
    assert rel(a_gpu, o.adjoint(c, gd, w.T)) < FP32_TOL
    assert F.device_status() == 0


@pytest.mark.skipif(os.environ.get("FFPAT_LONG_TESTS") != "1",
                    reason="about 15 minutes of oracle time on 16 cores; FFPAT_LONG_TESTS=1")
def test_config5_first_two_fb_iterations():
    """The first two iterations of the ramp-preconditioned Algorithm 8 on the
    large solve (N = 384, 180 angles, T = 1.5, 1 % noise, FP32-Kahan) against
    the oracle, iterates and history.  The step only scales the iterates, so
    a fixed s stands in for 1/L here (the oracle's power iteration would add
    40 wave solves)."""
    w, prec, c, h, prob = _config5_problem()
    g = as_input(add_noise(o.forward(c, h, w.T, w.n_angles), w.noise, w.noise_rel), prec)
    s = 1e-3
    hg, st, hist = F.fb_solve(prob, dev(c, prob), dev(g, prob), w.lam, s, 2)
    h_or, hist_or, k = o.fb(c, g, w.T, w.lam, s, 2, precond=1)
    assert st["iters_done"] == k == 2
    assert rel(host(hg), h_or) < FP32_TOL
    assert hist_dev(hist, hist_or) < FP32_TOL


# ------------------------------------------------- the two stencil kernels --

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,T", [(36, 0.4), (64, 0.3), (96, 0.12)])
def test_tma_stencil_matches_plain_and_oracle(n, T, prec):
    """The TMA-fed kernel and the plain 2.5D kernel compute the same steps;
    ragged tiles (36 = 64 - 28 in x, 36 = 4 x 8 + 4 in y) included."""
    c = as_input(random_speed(n, 900 + n), prec)
    h = as_input(random_volume(n, 901 + n), prec)
    prob = F.problem(n, T, 4, prec)
    outs = {}
    try:
        for path in (1, 2):
            F.set_stencil_path(path)
            outs[path] = (host(F.wave(prob, dev(c, prob), dev(h, prob))),
                          host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True)))
    finally:
        F.set_stencil_path(0)
    for a, b in zip(outs[1], outs[2]):
        assert rel(a, b) < (1e-14 if prec == F.FP64 else 1e-6)
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    kap = o.kappa(n, dt, c)
    assert rel(outs[2][0], o.wave(kap, h, nt)) < TOL[prec]
    assert rel(outs[2][1], o.wave_adjoint(kap, h, nt)) < TOL[prec]
    assert F.device_status() == 0


def test_tma_path_rejects_unaligned_sizes():
    prob = F.problem(33, 0.1, 4, F.FP32)
    try:
        F.set_stencil_path(2)
        with pytest.raises(F.FFPATError):
            F.wave(prob, dev(random_speed(33, 1), prob), dev(random_volume(33, 2), prob))
    finally:
        F.set_stencil_path(0)


@pytest.mark.parametrize("n,T", [(36, 0.4), (36, 0.41), (64, 0.3), (96, 0.21), (128, 0.05)])
def test_two_step_kahan_bit_identical(n, T):
    """Two FP32-Kahan steps per pass (temporal blocking) against one step per
    pass: the same per-point arithmetic, so W and W^T agree bit for bit, for
    even and odd step counts and ragged tiles; and both match the oracle."""
    prec = F.FP32_KAHAN
    c = as_input(random_speed(n, 1100 + n), prec)
    h = as_input(random_volume(n, 1101 + n), prec)
    prob = F.problem(n, T, 4, prec)
    outs = {}
    try:
        for path in (2, 3):
            F.set_stencil_path(path)
            outs[path] = (host(F.wave(prob, dev(c, prob), dev(h, prob))),
                          host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True)))
    finally:
        F.set_stencil_path(0)
    assert np.array_equal(outs[2][0], outs[3][0])
    assert np.array_equal(outs[2][1], outs[3][1])
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    assert rel(outs[3][0], o.wave(o.kappa(n, dt, c), h, nt)) < TOL[prec]
    assert F.device_status() == 0


@pytest.mark.parametrize("prec", [F.FP32_KAHAN, F.FP32])
@pytest.mark.parametrize("zc", [1, 3])
def test_two_step_many_items_per_cta(tmp_path, zc, prec):
    """The two-step passes with short z-ranges (FFPAT_ZCHUNK, in a child
    process): at N = 128 that is 688 or 2048 work items for 152 CTAs, so every
    CTA walks several items and re-arms its barriers between them; W and W^T
    stay bit for bit those of single steps."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n, T = 128, 0.05
    c = as_input(random_speed(n, 1300), F.FP32)
    h = as_input(random_volume(n, 1301), F.FP32)
    np.save(tmp_path / "c.npy", c.astype(np.float32))
    np.save(tmp_path / "h.npy", h.astype(np.float32))
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "from paper_1901_06503_gb300 import ffpat as F\n"
        f"c = torch.as_tensor(np.load({str(tmp_path / 'c.npy')!r}), device='cuda')\n"
        f"h = torch.as_tensor(np.load({str(tmp_path / 'h.npy')!r}), device='cuda')\n"
        f"prob = F.problem({n}, {T}, 4, {prec})\n"
        "out = []\n"
        "for path in (2, 3):\n"
        "    F.set_stencil_path(path)\n"
        "    out += [F.wave(prob, c, h).cpu().numpy(), F.wave(prob, c, h, transpose=True).cpu().numpy()]\n"
        "assert F.device_status() == 0\n"
        f"np.save({str(tmp_path / 'out.npy')!r}, np.stack(out))\n")
    env = dict(os.environ, FFPAT_ZCHUNK=str(zc))
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=300)
    w2, wt2, w3, wt3 = np.load(tmp_path / "out.npy").astype(np.float64)
    assert np.array_equal(w2, w3) and np.array_equal(wt2, wt3)
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    assert nt >= 4
    assert rel(w3, o.wave(o.kappa(n, dt, c), h, nt)) < FP32_TOL


@pytest.mark.parametrize("n,T", [(36, 0.4), (36, 0.41), (64, 0.3), (96, 0.21), (128, 0.05)])
def test_two_step_fp32_bit_identical(n, T):
    """Two FP32 three-term steps per pass against one step per pass (K1 and,
    through W^T = K^-1 W K, K3): bit-identical for even and odd step counts
    and ragged tiles, and matching the oracle."""
    prec = F.FP32
    c = as_input(random_speed(n, 1200 + n), prec)
    h = as_input(random_volume(n, 1201 + n), prec)
    prob = F.problem(n, T, 4, prec)
    outs = {}
    try:
        for path in (2, 3):
            F.set_stencil_path(path)
            outs[path] = (host(F.wave(prob, dev(c, prob), dev(h, prob))),
                          host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True)))
    finally:
        F.set_stencil_path(0)
    assert np.array_equal(outs[2][0], outs[3][0])
    assert np.array_equal(outs[2][1], outs[3][1])
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    assert rel(outs[3][0], o.wave(o.kappa(n, dt, c), h, nt)) < TOL[prec]
    assert F.device_status() == 0


@pytest.mark.parametrize("prec", [F.FP32, F.FP32_KAHAN])
@pytest.mark.parametrize("n,T", [(4, 0.9), (8, 0.5), (24, 0.004), (24, 0.03), (36, 0.41),
                                 (64, 0.3), (96, 0.21), (128, 0.05), (132, 0.03)])
def test_resident_loop_bit_identical(prec, n, T):
    """The whole time loop in one cooperative launch (registers and shared
    memory hold the per-point state, neighbour flags separate the steps)
    against one launch per step: W and W^T bit for bit, for one, two, odd and
    even step counts and ragged tiles; N = 132 does not fit the CTA slots, so
    forcing it fails and the automatic choice runs the step-by-step loop."""
    c = as_input(random_speed(n, 1300 + n), prec)
    h = as_input(random_volume(n, 1301 + n), prec)
    prob = F.problem(n, T, 4, prec)
    outs = {}
    try:
        for path in (2, 0, 4):
            F.set_stencil_path(path)
            if path == 4 and n > 128:
                with pytest.raises(F.FFPATError):
                    F.wave(prob, dev(c, prob), dev(h, prob))
                continue
            outs[path] = (host(F.wave(prob, dev(c, prob), dev(h, prob))),
                          host(F.wave(prob, dev(c, prob), dev(h, prob), transpose=True)))
    finally:
        F.set_stencil_path(0)
    for path in outs:
        assert np.array_equal(outs[2][0], outs[path][0]), path
        assert np.array_equal(outs[2][1], outs[path][1]), path
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    assert rel(outs[0][0], o.wave(o.kappa(n, dt, c), h, nt)) < TOL[prec]
    assert F.device_status() == 0


def test_resident_loops_on_two_streams():
    """Two resident time loops queued on two streams at once (each with its
    own workspace; each cooperative launch wants every SM) give the results
    of one stream, and no bounded wait runs out."""
    n, T, prec = 128, 1.2, F.FP32_KAHAN
    c = as_input(random_speed(n, 1500), prec)
    h1, h2 = as_input(random_volume(n, 1501), prec), as_input(random_volume(n, 1502), prec)
    prob = F.problem(n, T, 4, prec)
    cd, x1, x2 = dev(c, prob), dev(h1, prob), dev(h2, prob)
    ref1, ref2 = host(F.wave(prob, cd, x1)), host(F.wave(prob, cd, x2))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ws1, ws2 = F.workspace(prob), F.workspace(prob)
    o1, o2 = torch.empty_like(x1), torch.empty_like(x2)
    torch.cuda.synchronize()
    for _ in range(3):
        F.wave(prob, cd, x1, o1, ws=ws1, stream=s1)
        F.wave(prob, cd, x2, o2, ws=ws2, stream=s2)
    torch.cuda.synchronize()
    assert F.device_status() == 0
    assert np.array_equal(host(o1), ref1) and np.array_equal(host(o2), ref2)


@pytest.mark.parametrize("prec", [F.FP32, F.FP32_KAHAN])
@pytest.mark.parametrize("path", [0, 2, 3])
@pytest.mark.parametrize("T", [0.004, 0.1])
def test_wave_in_place(prec, path, T):
    """W with out = in (one step and several; resident loop, single steps and
    two steps per pass) equals the out-of-place result."""
    n = 24
    c = as_input(random_speed(n, 1400), prec)
    h = as_input(random_volume(n, 1401), prec)
    prob = F.problem(n, T, 4, prec)
    try:
        F.set_stencil_path(path)
        ref = host(F.wave(prob, dev(c, prob), dev(h, prob)))
        x = dev(h, prob)
        F.wave(prob, dev(c, prob), x, out=x)
        got = host(x)
    finally:
        F.set_stencil_path(0)
    assert np.array_equal(got, ref)


# ---------------------------------------------------- two-step method (Alg. 9) --

@pytest.mark.parametrize("prec", PRECS)
def test_fbp_and_two_step_fb(prec):
    w = config(1)
    c = as_input(w.c, prec)
    G = as_input(add_noise(o.forward(c, w.h, w.T, w.n_angles), w.noise, w.noise_rel), prec)
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    assert rel(host(F.fbp(prob, dev(G, prob))), o.fbp(G)) < (1e-10 if prec == F.FP64 else 2e-6)
    h_gpu, st, hist = F.fb_two_step(prob, dev(c, prob), dev(G, prob), w.lam, 0.5, 6)
    h_or, hist_or, k = o.fb_two_step(c, G, w.T, w.lam, 0.5, 6)
    assert st["iters_done"] == k == 6
    assert rel(host(h_gpu), h_or) < tol(prec)
    assert hist_dev(hist, hist_or, cols=(0,)) < hist_tol(prec)


def test_two_step_automatic_step():
    w = config(1)
    G = add_noise(o.forward(w.c, w.h, w.T, w.n_angles), w.noise, w.noise_rel)
    prob = F.problem(w.n, w.T, w.n_angles)
    _, st, _ = F.fb_two_step(prob, dev(w.c, prob), dev(G, prob), w.lam, 0.0, 1)
    # W is a polynomial in K L4 bounded by one in the kappa^-1-weighted norm
    assert 0.2 < st["opnorm_sq"] < 50 and abs(st["step"] * st["opnorm_sq"] - 1) < 1e-12


# ------------------------------------------ limited data chi_M, support chi_V --

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("precond", [0, 1])
def test_masked_fb(prec, precond):
    from paper_1901_06503_gb300.inputs import axis
    w, c, g, s = fb_case(prec, precond, n=20 if precond else None)
    xi = axis(w.n)
    mask = np.broadcast_to((np.abs(xi) > 0.25).astype(float), g.shape).copy()
    sup = np.zeros(c.shape)
    sup[3:-3, 3:-3, 3:-3] = 1.0
    prob = F.problem(w.n, w.T, w.n_angles, prec, precond)
    h_gpu, st, hist = F.fb_solve_masked(prob, dev(c, prob), dev(g, prob), w.lam, s, 6,
                                        mask=dev(mask, prob), support=dev(sup, prob))
    h_or, hist_or, k = o.fb_masked(c, g, w.T, w.lam, s, 6, mask=mask, support=sup,
                                   precond=precond)
    hg = host(h_gpu)
    assert st["iters_done"] == k == 6
    assert np.all(hg[sup == 0] == 0)
    assert rel(hg, h_or) < tol(prec)
    assert hist_dev(hist, hist_or) < hist_tol(prec)
