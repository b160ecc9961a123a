"""Seeded synthetic inputs: PA sources h, sound speeds c and noise draws.

This module holds no arithmetic of the reconstruction method itself; it only
draws the inputs.  The oracle side (tests) and the GPU side (tests, bench)
both take their inputs from here, so that they see identical arrays.

The paper's own phantom and trapping sound speed (Sec. 4.2, Fig. 1) are not
published as data, so every workload is synthetic: Gaussian blobs, balls with
Gaussian-smoothed edges and tubes along spline centrelines for h; a Gaussian
bump or a clipped Gaussian random field for c.  All arrays are float64 in
``[z][y][x]`` layout on the cell-centred grid of [-1, 1]^3.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy is present on both machines; keep a plain fallback for erfc anyway
    from scipy.special import erfc as _erfc
except Exception:  # pragma: no cover
    _erfc = np.vectorize(math.erfc)


def axis(n: int) -> np.ndarray:
    """Cell centres x_i = -1 + (i + 1/2) dx, dx = 2/n."""
    return -1.0 + (np.arange(n) + 0.5) * (2.0 / n)


def padded_axis(n: int, pad: int) -> np.ndarray:
    """Cell centres of the padded wave grid: the n cells of [-1, 1] plus pad
    cells of the same size dx = 2/n on either side (the same values as axis(n)
    on the image cells, bit for bit)."""
    return -1.0 + (np.arange(n + 2 * pad) - pad + 0.5) * (2.0 / n)


def extend_speed(c: np.ndarray, pad: int) -> np.ndarray:
    """A sound speed on the image grid continued to the padded wave grid by
    repeating its boundary values outwards."""
    return np.pad(np.asarray(c, dtype=np.float64), int(pad), mode="edge")


def _in_ball(rng: np.random.Generator, radius: float) -> np.ndarray:
    while True:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p <= radius * radius:
            return p


def _box(n: int, centre, reach: float):
    """Index slices of the grid points within `reach` (max-norm) of centre."""
    x = axis(n)
    sl = []
    for d in range(3):  # centre is (x, y, z); arrays are [z][y][x]
        c = centre[d]
        idx = np.nonzero(np.abs(x - c) <= reach)[0]
        if idx.size == 0:
            return None
        sl.append(slice(int(idx[0]), int(idx[-1]) + 1))
    return sl[2], sl[1], sl[0]


def gaussian_blobs(n, count, sigma, rmax, amp, rng) -> np.ndarray:
    x = axis(n)
    h = np.zeros((n, n, n))
    for _ in range(count):
        c = _in_ball(rng, rmax)
        a = rng.uniform(*amp)
        gz = np.exp(-((x - c[2]) ** 2) / (2 * sigma**2))
        gy = np.exp(-((x - c[1]) ** 2) / (2 * sigma**2))
        gx = np.exp(-((x - c[0]) ** 2) / (2 * sigma**2))
        h += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return h


def balls(n, count, radius, rmax, amp, rng) -> np.ndarray:
    """Balls with edges 1/2 erfc((|x - x_c| - R) / (sqrt(2) dx)), i.e. a step
    smoothed by a Gaussian of one voxel standard deviation."""
    x = axis(n)
    dx = 2.0 / n
    h = np.zeros((n, n, n))
    for _ in range(count):
        c = _in_ball(rng, rmax)
        R = rng.uniform(*radius)
        a = rng.uniform(*amp)
        box = _box(n, c, R + 5 * dx)
        if box is None:
            continue
        zs, ys, xs = box
        Z, Y, X = np.meshgrid(x[zs], x[ys], x[xs], indexing="ij")
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        h[zs, ys, xs] += a * 0.5 * _erfc((r - R) / (math.sqrt(2.0) * dx))
    return h


def _catmull_rom(pts: np.ndarray, samples: int) -> np.ndarray:
    out = []
    P = np.vstack([pts[0], pts, pts[-1]])
    for i in range(1, len(P) - 2):
        p0, p1, p2, p3 = P[i - 1], P[i], P[i + 1], P[i + 2]
        for t in np.linspace(0.0, 1.0, samples, endpoint=False):
            t2, t3 = t * t, t * t * t
            out.append(0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                              + (-p0 + 3 * p1 - 3 * p2 + p3) * t3))
    out.append(P[-2])
    return np.array(out)


def tubes(n, count, radius, rmax, amp, rng) -> np.ndarray:
    """Tubes of the given radius (erfc edge) around Catmull-Rom centrelines
    through 4 control points uniform in the ball of radius rmax."""
    x = axis(n)
    dx = 2.0 / n
    h = np.zeros((n, n, n))
    reach = radius + 5 * dx
    for _ in range(count):
        ctrl = np.array([_in_ball(rng, rmax) for _ in range(4)])
        a = rng.uniform(*amp)
        curve = _catmull_rom(ctrl, samples=max(64, 4 * n))
        dist = np.full((n, n, n), np.inf)
        for q in curve:
            box = _box(n, q, reach)
            if box is None:
                continue
            zs, ys, xs = box
            d = np.sqrt((x[xs][None, None, :] - q[0]) ** 2 + (x[ys][None, :, None] - q[1]) ** 2
                        + (x[zs][:, None, None] - q[2]) ** 2)
            np.minimum(dist[zs, ys, xs], d, out=dist[zs, ys, xs])
        m = np.isfinite(dist)
        h[m] += a * 0.5 * _erfc((dist[m] - radius) / (math.sqrt(2.0) * dx))
    return h


def speed_bump(n, amp, width, rmax, rng) -> np.ndarray:
    """c(x) = 1 + amp exp(-|x - x0|^2 / width^2), x0 uniform in the ball rmax."""
    x = axis(n)
    c0 = _in_ball(rng, rmax)
    r2 = ((x[None, None, :] - c0[0]) ** 2 + (x[None, :, None] - c0[1]) ** 2
          + (x[:, None, None] - c0[2]) ** 2)
    return 1.0 + amp * np.exp(-r2 / width**2)


def gaussian_random_field(n, corr_len, rng) -> np.ndarray:
    """White noise convolved (periodically) with a Gaussian of standard
    deviation corr_len / sqrt(2) -- covariance exp(-r^2 / (2 corr_len^2)) --
    then shifted and scaled to zero sample mean and unit sample std."""
    w = rng.standard_normal((n, n, n))
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=2.0 / n)
    kr = 2.0 * np.pi * np.fft.rfftfreq(n, d=2.0 / n)
    s = corr_len / math.sqrt(2.0)
    filt = np.exp(-0.5 * s * s * (k[:, None, None] ** 2 + k[None, :, None] ** 2
                                  + kr[None, None, :] ** 2))
    f = np.fft.irfftn(np.fft.rfftn(w) * filt, s=(n, n, n), axes=(0, 1, 2))
    f -= f.mean()
    f /= f.std()
    return f


@dataclasses.dataclass
class Workload:
    """One reconstruction problem: grid, physics, data shape and solver knobs."""

    name: str
    n: int
    T: float
    n_angles: int
    h: np.ndarray          # true PA source (float64)
    c: np.ndarray          # sound speed (float64, > 0)
    noise: np.ndarray      # standard normal draw of the data shape [theta][z][xi]
    noise_rel: float       # relative L2 noise level (0.01 = 1 %)
    iters: int
    lam: float = 1e-3
    precond: int = 0       # 0: Lambda = I, 1: ramp filter
    cfl: float = 0.3
    seed: int = 0

    @property
    def data_shape(self):
        return (self.n_angles, self.n, self.n)


def add_noise(clean: np.ndarray, noise: np.ndarray, rel: float) -> np.ndarray:
    """data = clean + sigma * noise with sigma = rel ||clean|| / sqrt(#data)."""
    sigma = rel * float(np.linalg.norm(clean.ravel())) / math.sqrt(clean.size)
    return clean + sigma * noise


def config(i: int, n: int | None = None, seed: int | None = None) -> Workload:
    """The five workloads: 1 small FP64 problem, 2 single 128^3 solve,
    3 differentiable 192^3 operator, 4 one request of the serving mix
    (its own seed), 5 large 384^3 preconditioned solve.  `n` rescales the grid
    with the same generator (used for oracle-sized copies)."""
    s = {1: 1, 2: 2, 3: 3, 4: 4, 5: 5}[i] if seed is None else seed
    rng = np.random.default_rng(s)
    if i == 1:
        n = n or 32
        h = gaussian_blobs(n, 3, 0.08, 0.5, (0.5, 1.0), rng)
        c = speed_bump(n, 0.2, 0.3, 0.3, rng)
        return Workload("fp64 one-step N=32^3, 24 angles, T=1", n, 1.0, 24, h, c,
                        rng.standard_normal((24, n, n)), 0.01, 10, 1e-3, 0, seed=s)
    if i == 2:
        n = n or 128
        h = balls(n, 20, (0.03, 0.1), 0.6, (0.2, 1.0), rng)
        c = np.clip(1.0 + 0.15 * gaussian_random_field(n, 0.25, rng), 0.8, 1.3)
        return Workload("single solve N=128^3, 90 angles, T=1.2", n, 1.2, 90, h, c,
                        rng.standard_normal((90, n, n)), 0.02, 100, 1e-3, 0, seed=s)
    if i == 3:
        n = n or 192
        h = balls(n, 50, (0.03, 0.1), 0.6, (0.2, 1.0), rng)
        c = speed_bump(n, 0.2, 0.3, 0.3, rng)
        return Workload("differentiable operator N=192^3, 90 angles, T=1", n, 1.0, 90, h, c,
                        rng.standard_normal((90, n, n)), 0.01, 1, 1e-3, 0, seed=s)
    if i == 4:
        n = n or int(rng.choice([64, 96, 128, 192]))
        nth = int(rng.choice([45, 90, 180]))
        T = float(rng.uniform(0.8, 1.4))
        iters = int(rng.integers(20, 61))
        h = gaussian_blobs(n, 3, 0.08, 0.5, (0.5, 1.0), rng)
        c = speed_bump(n, 0.2, 0.3, 0.3, rng)
        return Workload(f"serving request N={n}^3, {nth} angles, T={T:.3f}", n, T, nth, h, c,
                        rng.standard_normal((nth, n, n)), 0.01, iters, 1e-3, 0, seed=s)
    if i == 5:
        n = n or 384
        h = balls(n, 200, (0.03, 0.1), 0.6, (0.2, 1.0), rng)
        h += tubes(n, 5, 0.02, 0.6, (0.2, 1.0), rng)
        c = np.clip(1.0 + 0.25 * gaussian_random_field(n, 0.15, rng), 0.75, 1.4)
        return Workload("large solve N=384^3, 180 angles, T=1.5, ramp", n, 1.5, 180, h, c,
                        rng.standard_normal((180, n, n)), 0.01, 200, 1e-3, 1, seed=s)
    raise ValueError(i)


def random_volume(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((n, n, n))


def random_data(nth: int, n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((nth, n, n))


def random_speed(n: int, seed: int, lo: float = 0.8, hi: float = 1.25) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, n, n))
