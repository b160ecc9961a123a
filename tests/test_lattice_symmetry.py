"""The two symmetries of the ray-sample lattices (Sec. 3.1, the discrete X-ray
transform of eq. (4)) that the FP32 projection pair uses to serve four
angles with one evaluation, checked on the oracle's own sample points (CPU).

With N detectors and Ns samples, both spaced dx, and an even angle count 2h:
(1) the sample (k', m') of theta + 90 deg is the point (k, m) of theta's
    lattice with k' = m - (Ns - N)/2 and m' = (N + Ns)/2 - 1 - k;
(2) the sample (k, m') of 180 deg - theta is the mirror image x -> N-1-x of
    theta's point (k, Ns-1-m').
Positions are compared as continuous grid indices (corner + fraction); the
angles' own cos / sin differ from the rotated ones by rounding only.
"""
import numpy as np
import pytest

import oracle.oracle as o


def positions(n, nth, j, k, m):
    jkm = np.stack([np.full(k.size, j), k.ravel(), m.ravel()], axis=1)
    ij, f = o.sample_points(n, nth, jkm)
    return ij[:, 0] + f[:, 0], ij[:, 1] + f[:, 1]


@pytest.mark.parametrize("n,nth", [(16, 8), (24, 12), (40, 6)])
def test_rotation_by_90_samples_the_same_lattice(n, nth):
    ns = o.ray_samples(n)
    koff, mrot, h = (ns - n) // 2, (n + ns) // 2 - 1, nth // 2
    kp, mp = np.meshgrid(np.arange(n), np.arange(ns), indexing="ij")
    for j in range(h):
        xr, yr = positions(n, nth, j + h, kp, mp)
        x, y = positions(n, nth, j, mrot - mp, kp + koff)  # rows beyond 0..N-1 included
        assert np.max(np.abs(xr - x)) < 1e-9 and np.max(np.abs(yr - y)) < 1e-9, j


@pytest.mark.parametrize("n,nth", [(16, 8), (24, 12), (40, 6)])
def test_supplementary_angle_samples_the_mirror_image(n, nth):
    ns = o.ray_samples(n)
    k, mp = np.meshgrid(np.arange(n), np.arange(ns), indexing="ij")
    for j in range(1, nth):
        xs, ys = positions(n, nth, nth - j, k, mp)
        x, y = positions(n, nth, j, k, ns - 1 - mp)
        assert np.max(np.abs(xs - (n - 1 - x))) < 1e-9 and np.max(np.abs(ys - y)) < 1e-9, j


def test_four_angle_projection_from_one_lattice():
    """P of the four angles of a class, assembled from theta's lattice alone
    (row and column sums of the direct and the mirrored bilinear samples),
    equals the oracle's P of those angles."""
    n, nth = 24, 12
    ns = o.ray_samples(n)
    koff, h = (ns - n) // 2, nth // 2
    rng = np.random.default_rng(5)
    p = rng.standard_normal((3, n, n))
    want = o.project(np.concatenate([p, np.zeros((n - 3, n, n))]), nth)[:, :3]
    pad = np.zeros((3, n + 4, n + 4))
    pad[:, 2:n + 2, 2:n + 2] = p
    for j in (1, 2):
        kk, mm = np.meshgrid(np.arange(-koff, n + koff), np.arange(ns), indexing="ij")
        jkm = np.stack([np.full(kk.size, j), kk.ravel(), mm.ravel()], axis=1)
        ij, f = o.sample_points(n, nth, jkm)
        i0, j0, fx, fy = ij[:, 0], ij[:, 1], f[:, 0], f[:, 1]
        on = (i0 >= -1) & (i0 <= n - 1) & (j0 >= -1) & (j0 <= n - 1)
        i0c, j0c = np.clip(i0, -1, n - 1) + 2, np.clip(j0, -1, n - 1) + 2
        im = (n - 1 - np.clip(i0, -1, n - 1)) + 2  # mirror column of i0
        for pl in range(3):
            q = pad[pl]
            v = ((1 - fx) * (1 - fy) * q[j0c, i0c] + fx * (1 - fy) * q[j0c, i0c + 1]
                 + (1 - fx) * fy * q[j0c + 1, i0c] + fx * fy * q[j0c + 1, i0c + 1])
            vm = ((1 - fx) * (1 - fy) * q[j0c, im] + fx * (1 - fy) * q[j0c, im - 1]
                  + (1 - fx) * fy * q[j0c + 1, im] + fx * fy * q[j0c + 1, im - 1])
            v = np.where(on, v, 0.0).reshape(kk.shape)
            vm = np.where(on, vm, 0.0).reshape(kk.shape)
            dx = 2.0 / n
            got = {j: dx * v[koff:koff + n].sum(1),
                   j + h: dx * v.sum(0)[koff:koff + n],
                   nth - j: dx * vm[koff:koff + n].sum(1),
                   h - j: dx * vm.sum(0)[koff:koff + n]}
            for a, g in got.items():
                assert np.max(np.abs(g - want[a, pl])) < 1e-12 * max(1.0, np.abs(want[a, pl]).max()), (j, a, pl)
