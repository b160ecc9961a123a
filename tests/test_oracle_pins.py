"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed-form
solutions of the wave equation and of the X-ray transform, the Chebyshev
closed form of the leapfrog recurrence, exact reproduction of polynomials,
energy conservation, dense transposes, the filtered-backprojection identity
and the optimality conditions of the regularised functional.  Citations are to
Haltmeier, Zangerl, Nuster, Nguyen (2019).
"""
import math

import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300.inputs import (axis, padded_axis, random_data, random_speed,
                                           random_volume)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# ------------------------------------------------------------------ helpers --

def lap_from_wave(u, k0=0.1):
    """L4 u read off one oracle step: W with nt = 1 gives u + k0/2 L4 u."""
    kap = np.full(u.shape, k0)
    return (o.wave(kap, u, 1) - u) / (0.5 * k0)


def dense(op, n_in, shape_in):
    cols = []
    for i in range(n_in):
        e = np.zeros(n_in)
        e[i] = 1.0
        cols.append(np.asarray(op(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


def radial_gaussian(n, sigma):
    x = axis(n)
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    f = lambda s: np.exp(-s * s / (2 * sigma * sigma))  # noqa: E731
    return r, f


def spherical_solution(r, f, t):
    """3D radial d'Alembert solution of eq. (1)-(2) with c = 1, p_t(0) = 0."""
    return ((r - t) * f(r - t) + (r + t) * f(r + t)) / (2 * r)


# ------------------------------------------------------------ L4 and W_T --

def test_laplacian_exact_on_quintics():
    """Fourth-order central differences reproduce dx^2 * Laplacian exactly for
    polynomials of degree <= 5 (interior points, two away from the ghosts)."""
    n = 14
    dx = 2.0 / n
    x = axis(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = X**5 - 2 * X**2 * Y**3 + 0.5 * Y**4 * Z + Z**5 - 3 * X * Y * Z + 0.7 * Z**2
    lap = (20 * X**3 - 4 * Y**3 - 12 * X**2 * Y + 6 * Y**2 * Z + 20 * Z**3 + 1.4)
    got = lap_from_wave(u)[2:-2, 2:-2, 2:-2]
    want = dx * dx * lap[2:-2, 2:-2, 2:-2]
    assert np.max(np.abs(got - want)) < 1e-9 * np.max(np.abs(want))


def test_laplacian_dirichlet_principal_section():
    """Zero ghosts: the operator on an 8^3 box equals the 12^3 operator restricted
    to the inner 8^3 sub-box (principal section), and it is symmetric."""
    L8 = dense(lap_from_wave, 512, (8, 8, 8))
    L12 = dense(lap_from_wave, 12**3, (12, 12, 12))
    sub = np.zeros((12, 12, 12), bool)
    sub[2:10, 2:10, 2:10] = True
    sub = sub.ravel()
    assert np.max(np.abs(L12[np.ix_(sub, sub)] - L8)) < 1e-12
    assert np.max(np.abs(L8 - L8.T)) < 1e-12
    # the stencil reaches exactly two points along each axis
    nnz = np.count_nonzero(np.abs(L12[:, (6 * 12 + 6) * 12 + 6]) > 1e-12)
    assert nnz == 13


def test_wave_chebyshev_closed_form():
    """p^n = T_n(I + K L4 / 2) h: the leapfrog with the zero-velocity start step
    is the Chebyshev polynomial of the first kind, evaluated here through the
    eigen-decomposition of the symmetrised S = I + K^1/2 L4 K^1/2 / 2
    (T_n(cos a) = cos(n a))."""
    n = 8
    L = dense(lap_from_wave, n**3, (n, n, n))
    kap = np.random.default_rng(7).uniform(0.02, 0.06, n**3)
    sk = np.sqrt(kap)
    S = np.eye(n**3) + 0.5 * sk[:, None] * L * sk[None, :]
    lam, Q = np.linalg.eigh(S)
    assert lam.min() > -1 and lam.max() <= 1 + 1e-12
    for nt in (1, 2, 5, 13):
        Tn = np.cos(nt * np.arccos(np.clip(lam, -1, 1)))
        W_closed = (sk[:, None] * (Q * Tn) @ Q.T) / sk[None, :]
        W_or = dense(lambda h: o.wave(kap.reshape(n, n, n), h, nt), n**3, (n, n, n))
        assert np.max(np.abs(W_or - W_closed)) < 1e-11
        Wt = dense(lambda g: o.wave_adjoint(kap.reshape(n, n, n), g, nt), n**3, (n, n, n))
        assert np.max(np.abs(Wt - W_or.T)) < 1e-13


def test_wave_spherical_solution_space_order():
    """Closed-form radial solution, c = 1 (d'Alembert for r p): with a small
    time step the error is the spatial one, fourth order."""
    errs = []
    for n in (48, 96):
        r, f = radial_gaussian(n, 0.08)
        nt, dt = o.time_steps(n, 0.3, 0.02, 1.0)
        p = o.wave(o.kappa(n, dt, np.ones((n, n, n))), f(r), nt)
        errs.append(rel(p, spherical_solution(r, f, 0.3)))
    order = math.log2(errs[0] / errs[1])
    assert errs[1] < 3e-3
    assert 3.5 < order < 4.6, (errs, order)


def test_wave_time_order_two():
    """Leapfrog plus the second-order start step: successive differences under
    halving of the CFL number shrink by 4 (second order in time)."""
    n = 48
    r, f = radial_gaussian(n, 0.08)
    ps = []
    for cfl in (0.4, 0.2, 0.1):
        nt, dt = o.time_steps(n, 0.3, cfl, 1.0)
        ps.append(o.wave(o.kappa(n, dt, np.ones((n, n, n))), f(r), nt))
    ratio = np.linalg.norm(ps[0] - ps[1]) / np.linalg.norm(ps[1] - ps[2])
    assert 3.6 < ratio < 4.5
    # and the standard CFL run is close to the closed form
    assert rel(ps[1], spherical_solution(r, f, 0.3)) < 0.02


def test_leapfrog_energy_conserved():
    """E^{n+1/2} = <K^-1 (p^{n+1} - p^n), p^{n+1} - p^n> - <L4 p^{n+1}, p^n> is
    invariant under the recurrence, with a variable sound speed, and positive
    under the CFL bound."""
    n = 12
    rng = np.random.default_rng(3)
    kap = rng.uniform(0.03, 0.09, (n, n, n))
    h = random_volume(n, 4)
    energies = []
    prev = o.wave(kap, h, 1)
    for nt in range(2, 30):
        cur = o.wave(kap, h, nt)
        d = cur - prev
        e = np.sum(d * d / kap) - np.sum(lap_from_wave(cur) * prev)
        energies.append(e)
        prev = cur
    energies = np.array(energies)
    assert energies.min() > 0
    assert np.max(np.abs(energies - energies[0])) < 1e-12 * abs(energies[0])


def test_time_steps_rounding():
    """Nt: smallest count with dt <= cfl dx / c_max; exact ratios do not gain a step."""
    assert o.time_steps(384, 1.5, 0.3, 1.4)[0] == 1344
    assert o.time_steps(32, 1.0, 0.3, 1.2)[0] == 64
    nt, dt = o.time_steps(128, 1.2, 0.3, 1.3)
    assert nt == 333 and abs(dt * nt - 1.2) < 1e-15
    assert o.time_steps(16, 1e-6, 0.3, 1.0)[0] == 1


# ------------------------------------------------------- X-ray transform --

def gaussian3(n, x0, sigma, amp=1.0):
    x = axis(n)
    return amp * (np.exp(-((x - x0[2]) ** 2) / (2 * sigma**2))[:, None, None]
                  * np.exp(-((x - x0[1]) ** 2) / (2 * sigma**2))[None, :, None]
                  * np.exp(-((x - x0[0]) ** 2) / (2 * sigma**2))[None, None, :])


def test_projection_axis_aligned_sums():
    """At theta = 0 the rays run along y through the x cell centres and the
    samples hit the y centres, so P is ds times column sums; at theta = pi/2
    it is ds times row sums (orientation of xi and of the (x, y) axes)."""
    n, nth = 16, 4
    p = random_volume(n, 11)
    g = o.project(p, nth)
    ds = 2.0 / n
    assert np.max(np.abs(g[0] - ds * p.sum(axis=1))) < 1e-12
    assert np.max(np.abs(g[2] - ds * p.sum(axis=2))) < 1e-12


def test_projection_of_gaussian_closed_form():
    """X[A e^{-|x-x0|^2/2s^2}](theta, xi, z) = A sqrt(2 pi) s
    e^{-(xi - <theta, x0>)^2/2s^2} e^{-(z - z0)^2/2s^2}, eq. (4); error O(dx^2)."""
    x0, sigma, nth = (0.13, -0.21, 0.05), 0.1, 7
    errs = []
    for n in (32, 64, 128):
        x = axis(n)
        g = o.project(gaussian3(n, x0, sigma, 0.8), nth)
        th = np.pi * np.arange(nth) / nth
        proj = x0[0] * np.cos(th) + x0[1] * np.sin(th)
        want = (0.8 * math.sqrt(2 * math.pi) * sigma
                * np.exp(-((x[None, None, :] - proj[:, None, None]) ** 2) / (2 * sigma**2))
                * np.exp(-((x[None, :, None] - x0[2]) ** 2) / (2 * sigma**2)))
        errs.append(rel(g, want))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


def test_sample_tables():
    """Ray samples: 2 ceil(N / sqrt 2) of them; angles pi j / n_angles."""
    assert o.ray_samples(32) == 46 and o.ray_samples(128) == 182 and o.ray_samples(384) == 544
    cs, sn = o.angles(6)
    th = np.pi * np.arange(6) / 6
    assert np.array_equal(cs, np.cos(th)) and np.array_equal(sn, np.sin(th))
    ij, f = o.sample_points(16, 4, [[0, 3, 0], [0, 3, 11]])
    # theta = 0: x = xi_3 -> grid index 3 (up to one rounding), y = s_m
    gx = ij[:, 0] + f[:, 0]
    assert np.allclose(gx, 3.0, atol=1e-12)
    ns = o.ray_samples(16)
    assert np.allclose(ij[:, 1] + f[:, 1], np.array([0, 11]) - ns // 2 + 8, atol=1e-12)


def test_project_rays_is_project():
    n, nth = 12, 5
    p = random_volume(n, 13)
    g = o.project(p, nth)
    jlk = np.array([[j, l, k] for j in range(nth) for l in range(n) for k in range(n)])
    assert np.array_equal(o.project_rays(p, nth, jlk), g.ravel())


def test_projection_transpose_dense():
    """P^T is the exact matrix transpose of P (8^3 grid, 6 angles)."""
    n, nth = 8, 6
    P = dense(lambda p: o.project(p, nth), n**3, (n, n, n))
    PT = dense(lambda g: o.backproject(g, n), nth * n * n, (nth, n, n))
    assert np.max(np.abs(PT - P.T)) < 1e-14


# ------------------------------------------------------------- Lambda --

def test_ramp_taps_frequency_response():
    """The taps realise |omega| / (4 pi) on the detector spacing: the DTFT
    sum_d t_d cos(omega d dxi) equals |omega| / (4 pi) for |omega| <= pi / dxi."""
    n = 64
    dxi = 2.0 / n
    d = np.arange(1, 200001)
    taps = np.where(d % 2 == 1, -1.0 / (2 * np.pi**2 * d.astype(float) ** 2 * dxi), 0.0)
    for i, dd in enumerate((1, 2, 3, 7, 8)):
        assert o.ramp_tap(n, dd) == taps[dd - 1] or abs(o.ramp_tap(n, dd) - taps[dd - 1]) < 1e-15
    t0 = o.ramp_tap(n, 0)
    for w in (0.3, 5.0, 40.0, 90.0):
        resp = t0 + 2 * np.sum(taps * np.cos(w * d * dxi))
        assert abs(resp - w / (4 * np.pi)) < 2e-5 * max(1.0, w / (4 * np.pi)) + 2e-5


def test_ramp_matches_fourier_filter():
    """Lambda applied to a well-sampled Gaussian row equals the Fourier-domain
    filter |omega| / (4 pi) (computed with a heavily padded FFT)."""
    n, nth = 64, 2
    x = axis(n)
    row = np.exp(-((x - 0.1) ** 2) / (2 * 0.08**2))
    r = np.tile(row, (nth, n, 1))
    got = o.ramp(r)[0, 0]
    pad = 64
    m = n * pad
    big = np.zeros(m)
    big[:n] = row
    w = 2 * np.pi * np.fft.fftfreq(m, d=2.0 / n)
    want = np.real(np.fft.ifft(np.fft.fft(big) * np.abs(w) / (4 * np.pi)))[:n]
    assert rel(got, want) < 1e-3


def test_ramp_symmetric():
    n, nth = 10, 3
    R = dense(o.ramp, nth * n * n, (nth, n, n))
    assert np.max(np.abs(R - R.T)) < 1e-13
    assert np.linalg.eigvalsh(R).min() > -1e-12


def test_fbp_identity():
    """X* Lambda = X^{-1} (Sec. 3.1): (2 pi / (n_angles dx)) P^T Lambda P h ~ h
    for a smooth z-constant h (backprojection over S^1 is twice [0, pi))."""
    n, nth = 96, 144
    x = axis(n)
    plane = (np.exp(-((x[:, None] - 0.1) ** 2 + (x[None, :] + 0.15) ** 2) / (2 * 0.15**2))
             + 0.5 * np.exp(-((x[:, None] + 0.3) ** 2 + (x[None, :] - 0.2) ** 2) / (2 * 0.1**2)))
    h = np.broadcast_to(plane, (n, n, n)).copy()
    g = o.project(h, nth)
    rec = (2 * np.pi / (nth * (2.0 / n))) * o.backproject(o.ramp(g), n)
    inner = (slice(n // 2, n // 2 + 1), slice(12, -12), slice(12, -12))
    assert rel(rec[inner], h[inner]) < 0.03


# ----------------------------------------------------- composite operator --

@pytest.mark.parametrize("T", [0.004, 0.009, 0.5])
def test_dot_product(T):
    """<A h, g> = <h, A^T g> to 1e-12 (includes Nt = 1 and Nt = 2)."""
    n, nth = 12, 5
    c = random_speed(n, 21)
    h = random_volume(n, 22)
    g = random_data(nth, n, 23)
    Ah = o.forward(c, h, T, nth)
    Atg = o.adjoint(c, g, T)
    lhs, rhs = float(np.sum(Ah * g)), float(np.sum(h * Atg))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ah) * np.linalg.norm(g)


def test_dalembert_plane_integrals():
    """Plane integrals of p obey the 1D wave equation (Sec. 2.2):
    sum_l dz g[j, l, k] ~ 1/2 (Rh(theta, xi - cT) + Rh(theta, xi + cT)), with
    Rh the plane integral A 2 pi s^2 e^{-(xi - <theta, x0>)^2 / 2 s^2} of a
    Gaussian blob (c = 1, nothing reaches the box boundary)."""
    x0, sigma, amp, T, nth = (0.07, -0.05, 0.02), 0.08, 0.9, 0.3, 5
    errs = []
    for n in (32, 64):
        x = axis(n)
        h = gaussian3(n, x0, sigma, amp)
        g = o.forward(np.ones((n, n, n)), h, T, nth)
        got = g.sum(axis=1) * (2.0 / n)
        th = np.pi * np.arange(nth) / nth
        pr = x0[0] * np.cos(th) + x0[1] * np.sin(th)
        Rh = lambda s: amp * 2 * np.pi * sigma**2 * np.exp(-((s - pr[:, None]) ** 2) / (2 * sigma**2))  # noqa
        want = 0.5 * (Rh(x[None, :] - T) + Rh(x[None, :] + T))
        errs.append(rel(got, want))
    assert errs[1] < 1.5e-2 and 3.5 < errs[0] / errs[1] < 4.6, errs


# ---------------------------------------------------------- Algorithm 8 --

def dense_A(n, nth, c, T):
    return dense(lambda h: o.forward(c, h, T, nth), n**3, (n, n, n))


def test_power_iteration_matches_dense_eigenvalue():
    n, nth, T = 6, 4, 0.6
    c = random_speed(n, 31)
    A = dense_A(n, nth, c, T)
    for precond in (0, 1):
        if precond:
            LA = dense(lambda h: o.ramp(o.forward(c, h, T, nth)), n**3, (n, n, n))
        else:
            LA = A
        lam_max = np.linalg.eigvalsh(A.T @ LA).max()
        v0 = random_volume(n, 32)
        est = o.power(c, v0, T, nth, precond=precond, iters=400)
        assert abs(est - lam_max) < 1e-6 * lam_max


def test_fb_first_step_and_prox():
    """From h_0 = 0 one step of Algorithm 8 is max(s A^T g - s lambda, 0)
    (gradient of 1/2||Ah - g||^2 at 0 is -A^T g; prox of s lambda (l1 + i_{>=0}))."""
    n, nth, T = 10, 6, 0.5
    c = random_speed(n, 41)
    g = random_data(nth, n, 42)
    s, lam = 0.05, 0.3
    h1, stats, k = o.fb(c, g, T, lam, s, 1)
    want = np.maximum(s * o.adjoint(c, g, T) - s * lam, 0.0)
    assert k == 1 and np.max(np.abs(h1 - want)) < 1e-13 * max(1.0, np.abs(want).max())
    assert abs(stats[0, 1] - np.linalg.norm(g)) < 1e-12 * np.linalg.norm(g)
    assert abs(stats[0, 0] - 0.5 * np.sum(g * g)) < 1e-12 * np.sum(g * g)


def test_fb_kkt_at_fixed_point():
    """After many FB iterations h is a minimiser of 1/2 <Lambda(Ah - g), Ah - g>
    + lambda (||h||_1 + i_{>=0}): grad_i + lambda = 0 where h_i > 0 and
    grad_i + lambda >= 0 where h_i = 0 (for both Lambda = I and the ramp)."""
    n, nth, T = 6, 8, 0.5
    c = random_speed(n, 51)
    rng = np.random.default_rng(52)
    h_true = np.maximum(rng.standard_normal((n, n, n)), 0)
    for precond in (0, 1):
        g = o.forward(c, h_true, T, nth)
        A = dense_A(n, nth, c, T)
        LA = dense(lambda h: o.ramp(o.forward(c, h, T, nth)), n**3, (n, n, n)) if precond else A
        H = A.T @ LA
        Lmax = np.linalg.eigvalsh(H).max()
        lam = 0.02 * float(np.abs(A.T @ (o.ramp(g) if precond else g).ravel()).max())
        h, stats, k = o.fb(c, g, T, lam, 1.0 / Lmax, 6000, precond=precond)
        hr = h.ravel()
        grad = H @ hr - LA.T @ g.ravel()
        pos = hr > 1e-9
        # a wrong sign, prox or threshold leaves violations of order lambda
        assert pos.any() and (~pos).any()
        assert np.max(np.abs(grad[pos] + lam)) < 1e-3 * lam
        assert np.min(grad[~pos] + lam) > -1e-3 * lam
        obj = stats[:, 0]
        assert np.all(np.diff(obj) <= 1e-12 * abs(obj[0]))


def test_fb_tolerance_stops_early():
    n, nth, T = 6, 4, 0.4
    c = random_speed(n, 61)
    g = random_data(nth, n, 62)
    L = o.power(c, random_volume(n, 63), T, nth, iters=50)
    h, stats, k = o.fb(c, g, T, 1e-3, 1.0 / L, 500, tol=1e-3)
    assert 1 < k < 500 and stats[-1, 2] < 1e-3 and np.all(stats[:-1, 2] >= 1e-3)


# ------------------------------------------------- gradient with respect to c --

def test_grad_c_matches_central_differences():
    """d/dc <w, A(c) h> against central differences of the oracle forward along
    random directions (dt frozen at its value for c: the perturbation keeps
    max c and hence Nt fixed)."""
    n, nth, T = 10, 5, 0.5
    rng = np.random.default_rng(71)
    c = random_speed(n, 72, 0.9, 1.1)
    c[0, 0, 0] = 1.2  # the maximum, never perturbed
    h = random_volume(n, 73)
    w = random_data(nth, n, 74)
    gh, gc = o.grad(c, h, w, T)
    assert np.allclose(gh, o.adjoint(c, w, T), rtol=0, atol=1e-12 * np.abs(gh).max())
    eps = 1e-5
    for _ in range(6):
        d = rng.standard_normal((n, n, n))
        d[0, 0, 0] = 0.0
        fp = np.sum(w * o.forward(c + eps * d, h, T, nth))
        fm = np.sum(w * o.forward(c - eps * d, h, T, nth))
        fd = (fp - fm) / (2 * eps)
        an = float(np.sum(gc * d))
        assert abs(fd - an) < 1e-6 * max(abs(fd), 1e-3)


def test_grad_c_single_step_closed_form():
    """Nt = 1: A h = P (h + kappa/2 L4 h), so d/dc_i = (P^T w)_i (L4 h)_i kappa_i / c_i."""
    n, nth = 8, 4
    c = random_speed(n, 81, 0.9, 1.1)
    T = 0.3 * (2.0 / n) / c.max() * 0.99
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    assert nt == 1
    h = random_volume(n, 82)
    w = random_data(nth, n, 83)
    kap = o.kappa(n, dt, c)
    _, gc = o.grad(c, h, w, T)
    want = o.backproject(w, n) * lap_from_wave(h) * kap / c
    assert np.allclose(gc, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


# ------------------------------------------------------ two-step method (Alg. 9) --

def test_fbp_is_the_scaled_filtered_backprojection():
    """fbp = (2 pi / (n_angles dx)) P^T Lambda (the discrete X* Lambda of Sec. 3.1,
    whose accuracy the FBP identity pin checks)."""
    n, nth = 12, 9
    G = random_data(nth, n, 91)
    want = (2 * np.pi / (nth * (2.0 / n))) * o.backproject(o.ramp(G), n)
    assert np.allclose(o.fbp(G), want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_two_step_first_iterate_and_kkt():
    """Algorithm 9: from h_0 = 0 the first iterate is max(s W^T g - s lambda, 0)
    with g = X^{-1} G; at the fixed point the KKT conditions of
    1/2 ||W h - g||^2 + lambda (||h||_1 + i_{>=0}) hold (dense W at 6^3)."""
    n, nth, T = 6, 8, 0.5
    c = random_speed(n, 92)
    G = random_data(nth, n, 93)
    g = o.fbp(G)
    nt, dt = o.time_steps(n, T, 0.3, c.max())
    kap = o.kappa(n, dt, c)
    s, lam = 0.3, 0.05
    h1, st, k = o.fb_two_step(c, G, T, lam, s, 1)
    want = np.maximum(s * o.wave_adjoint(kap, g, nt) - s * lam, 0.0)
    assert np.max(np.abs(h1 - want)) < 1e-13 * max(1.0, np.abs(want).max())
    Wd = dense(lambda h: o.wave(kap, h, nt), n**3, (n, n, n))
    H = Wd.T @ Wd
    Lmax = np.linalg.eigvalsh(H).max()
    lam = 0.02 * float(np.abs(Wd.T @ g.ravel()).max())
    h, st, k = o.fb_two_step(c, G, T, lam, 1.0 / Lmax, 4000)
    hr = h.ravel()
    grad = H @ hr - Wd.T @ g.ravel()
    pos = hr > 1e-9
    assert pos.any() and (~pos).any()
    assert np.max(np.abs(grad[pos] + lam)) < 1e-3 * lam
    assert np.min(grad[~pos] + lam) > -1e-3 * lam


# ------------------------------------------ limited data chi_M, support chi_V --

def _masks(n, nth, a=0.3, box=(2, -2)):
    xi = axis(n)
    mask = np.broadcast_to((np.abs(xi) > a).astype(float), (nth, n, n)).copy()
    sup = np.zeros((n, n, n))
    lo, hi = box
    sup[lo:hi, lo:hi, lo:hi] = 1.0
    return mask, sup


def test_masked_fb_reduces_and_first_step():
    """With all-ones masks the masked FB is Algorithm 8; from h_0 = 0 one masked
    step is chi_V max(s A^T chi g - s lambda, 0) (Lambda = I)."""
    n, nth, T = 10, 6, 0.5
    c = random_speed(n, 95)
    g = random_data(nth, n, 96)
    h_a, st_a, _ = o.fb(c, g, T, 1e-3, 0.05, 3)
    h_b, st_b, _ = o.fb_masked(c, g, T, 1e-3, 0.05, 3, mask=np.ones((nth, n, n)),
                               support=np.ones((n, n, n)))
    assert np.array_equal(h_a, h_b) and np.array_equal(st_a, st_b)
    mask, sup = _masks(n, nth)
    s, lam = 0.05, 0.2
    h1, _, _ = o.fb_masked(c, g, T, lam, s, 1, mask=mask, support=sup)
    want = sup * np.maximum(s * o.adjoint(c, mask * g, T) - s * lam, 0.0)
    assert np.max(np.abs(h1 - want)) < 1e-13 * max(1.0, np.abs(want).max())


def test_masked_fb_kkt():
    """KKT of 1/2 <chi Lambda chi (Ah - g), Ah - g> + lambda (||h||_1 + i_{>=0} + i_V)
    at the fixed point (dense A at 6^3, ramp preconditioner, |xi| > a data)."""
    n, nth, T = 6, 8, 0.5
    c = random_speed(n, 97)
    rng = np.random.default_rng(98)
    h_true = np.maximum(rng.standard_normal((n, n, n)), 0)
    g = o.forward(c, h_true, T, nth)
    mask, sup = _masks(n, nth, a=0.2, box=(1, -1))
    A = dense_A(n, nth, c, T)
    M = mask.ravel()
    LA = dense(lambda h: mask * o.ramp(mask * o.forward(c, h, T, nth)), n**3, (n, n, n))
    H = A.T @ LA
    inside = sup.ravel() > 0
    Hs = H[np.ix_(inside, inside)]
    Lmax = np.linalg.eigvalsh(0.5 * (Hs + Hs.T)).max()
    b = A.T @ (M * o.ramp(mask * g).ravel())
    lam = 0.02 * float(np.abs(b[inside]).max())
    h, st, k = o.fb_masked(c, g, T, lam, 1.0 / Lmax, 6000, mask=mask, support=sup, precond=1)
    hr = h.ravel()
    assert np.all(hr[~inside] == 0)
    grad = H @ hr - b
    pos = (hr > 1e-9) & inside
    zero = (hr <= 1e-9) & inside
    assert pos.any() and zero.any()
    assert np.max(np.abs(grad[pos] + lam)) < 1e-3 * lam
    assert np.min(grad[zero] + lam) > -1e-3 * lam


# ------------------------------------------ padded wave grid (Sec. 5 setup) --

def test_padded_wave_matches_free_space_solution():
    """With the wave grid padded (V_T larger than the box V) the outgoing
    spherical wave of an off-centre Gaussian travels past the box faces: on the
    whole wave grid W_T E follows the free-space radial solution (c = 1), while
    the box-sized operator (Dirichlet walls at the faces) carries the wave
    reflected back into the box."""
    x0, sigma, T = 0.45, 0.08, 0.75
    errs = []
    for n in (32, 64):
        pad = n // 2
        f = lambda s: np.exp(-s * s / (2 * sigma * sigma))  # noqa: E731
        x = axis(n)
        r = np.sqrt((x[None, None, :] - x0) ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2)
        xw = padded_axis(n, pad)
        rw = np.sqrt((xw[None, None, :] - x0) ** 2 + xw[None, :, None] ** 2
                     + xw[:, None, None] ** 2)
        got = o.wave_pad(np.ones((n + 2 * pad,) * 3), f(r), T, pad)
        assert got.shape == (n + 2 * pad,) * 3
        errs.append(rel(got, spherical_solution(rw, f, T)))
        if n == 64:
            walls = rel(o.wave_pad(np.ones((n,) * 3), f(r), T, 0), spherical_solution(r, f, T))
            inbox = rel(got[pad:-pad, pad:-pad, pad:-pad], spherical_solution(r, f, T))
    # N = 32 is coarse for sigma = 0.08 (pre-asymptotic): ask for at least
    # second-order-like decay
    assert errs[1] < 2e-2 and errs[0] / errs[1] > 3.5, errs
    assert walls > 10 * inbox, (walls, inbox)


def test_padded_dalembert_past_the_box():
    """The 1D reduction of Sec. 2.2 on the padded grid: the plane integrals
    sum_l dz g[j, l, k] of the data of the whole wave grid follow
    1/2 (Rh(xi - T) + Rh(xi + T)) with xi on the padded detector line, also
    once the waves have left the box (T = 0.8 here, c = 1)."""
    x0, sigma, amp, T, nth = (0.3, -0.2, 0.1), 0.08, 0.9, 0.8, 5
    errs = []
    for n in (32, 64):
        pad = n // 2
        x = axis(n)
        gz = np.exp(-((x - x0[2]) ** 2) / (2 * sigma**2))
        gy = np.exp(-((x - x0[1]) ** 2) / (2 * sigma**2))
        gx = np.exp(-((x - x0[0]) ** 2) / (2 * sigma**2))
        h = amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        g = o.forward(np.ones((n + 2 * pad,) * 3), h, T, nth, pad=pad)
        assert g.shape == (nth, n + 2 * pad, n + 2 * pad)
        got = g.sum(axis=1) * (2.0 / n)
        th = np.pi * np.arange(nth) / nth
        pr = x0[0] * np.cos(th) + x0[1] * np.sin(th)
        Rh = lambda s: amp * 2 * np.pi * sigma**2 * np.exp(-((s - pr[:, None]) ** 2) / (2 * sigma**2))  # noqa
        xi = padded_axis(n, pad)
        errs.append(rel(got, 0.5 * (Rh(xi[None, :] - T) + Rh(xi[None, :] + T))))
    assert errs[1] < 1.5e-2 and 3.0 < errs[0] / errs[1] < 5.0, errs


def test_padded_operator_transpose_dense():
    """The padded A (zero-extend, W_T on the wave grid, P of the wave grid)
    and its transpose, as dense matrices (5^3 box, 2 cells of padding, variable
    c); likewise W_T E and E^T W_T^T."""
    n, pad, nth, T = 5, 2, 4, 0.5
    nw = n + 2 * pad
    c = random_speed(nw, 131)
    A = dense(lambda h: o.forward(c, h, T, nth, pad=pad), n**3, (n, n, n))
    At = dense(lambda g: o.adjoint(c, g, T, pad=pad), nth * nw * nw, (nth, nw, nw))
    assert A.shape == (nth * nw * nw, n**3)
    assert np.max(np.abs(At - A.T)) <= 1e-13 * np.abs(A).max()
    W = dense(lambda h: o.wave_pad(c, h, T, pad), n**3, (n, n, n))
    Wt = dense(lambda u: o.wave_pad(c, u, T, pad, transpose=True), nw**3, (nw, nw, nw))
    assert np.max(np.abs(Wt - W.T)) <= 1e-13 * np.abs(W).max()


def test_padded_projection_is_the_scaled_grid_projection():
    """P on a grid of cells of size 2 / nimg is the same index geometry as on
    the unit box, with samples of length 2 / nimg: P_nimg = (ng / nimg) P_ng;
    likewise Lambda_nimg = (nimg / ng) Lambda_ng (taps ~ 1 / dxi); the
    filtered backprojection scales by nimg / ng, so that as an inverse of P it
    is unchanged: FBP_nimg P_nimg = FBP_ng P_ng."""
    ng, nimg, nth = 14, 10, 6
    p = random_volume(ng, 141)
    assert np.max(np.abs(o.project(p, nth, nimg) - (ng / nimg) * o.project(p, nth))) < 1e-13
    r = random_data(nth, ng, 142)
    assert np.max(np.abs(o.ramp(r, nimg) - (nimg / ng) * o.ramp(r))) < 1e-12
    assert np.max(np.abs(o.backproject(r, ng, nimg) - (ng / nimg) * o.backproject(r, ng))) < 1e-13
    assert np.max(np.abs(o.fbp(r, nimg) - (nimg / ng) * o.fbp(r))) < 1e-12
    a, b = o.fbp(o.project(p, nth, nimg), nimg), o.fbp(o.project(p, nth))
    assert np.max(np.abs(a - b)) < 1e-12 * np.abs(b).max()


def test_padding_past_the_domain_of_dependence():
    """The stencil reaches two cells per step, so once the padding has at least
    Nt cells the walls cannot reach the box within Nt steps: the box part of
    W_T E h is then the same, bit for bit, for any larger padding (c a smooth
    function of position, the same on the shared cells); thin padding changes it."""
    n, T = 8, 0.25
    h = random_volume(n, 133)

    def speed(pad):
        x = padded_axis(n, pad)
        r2 = x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2
        return 1.0 + 0.2 * np.exp(-r2 / 0.09)

    def box(u, pad):
        return u[pad:pad + n, pad:pad + n, pad:pad + n]

    nt, _ = o.time_steps(n, T, 0.3, float(speed(0).max()))
    assert nt >= 3
    w1 = box(o.wave_pad(speed(nt), h, T, nt), nt)
    w2 = box(o.wave_pad(speed(nt + 3), h, T, nt + 3), nt + 3)
    assert np.array_equal(w1, w2)
    assert not np.array_equal(box(o.wave_pad(speed(1), h, T, 1), 1), w1)
    assert np.array_equal(padded_axis(n, 0), axis(n))
    assert np.array_equal(padded_axis(n, 3)[3:-3], axis(n))


def test_padded_fb_kkt():
    """Algorithm 8 on the padded operator reaches the KKT point of
    1/2 ||A h - g||^2 + lambda (||h||_1 + i_{>=0}) (dense padded A at 5^3)."""
    n, pad, nth, T = 5, 2, 6, 0.6
    c = random_speed(n + 2 * pad, 137)
    rng = np.random.default_rng(138)
    g = o.forward(c, np.maximum(rng.standard_normal((n, n, n)), 0), T, nth, pad=pad)
    A = dense(lambda h: o.forward(c, h, T, nth, pad=pad), n**3, (n, n, n))
    H = A.T @ A
    L = np.linalg.eigvalsh(H).max()
    assert abs(o.power(c, random_volume(n, 139), T, nth, iters=400, pad=pad) - L) < 1e-6 * L
    b = A.T @ g.ravel()
    lam = 0.02 * float(np.abs(b).max())
    h, st, k = o.fb_masked(c, g, T, lam, 1.0 / L, 6000, pad=pad)
    hr = h.ravel()
    grad = H @ hr - b
    pos, zero = hr > 1e-9, hr <= 1e-9
    assert pos.any() and zero.any()
    assert np.max(np.abs(grad[pos] + lam)) < 1e-3 * lam
    assert np.min(grad[zero] + lam) > -1e-3 * lam


# ------------------------- gradient regulariser R = 1/2 |grad h|^2 (Sec. 5) --

def neumann_dtd(h):
    """D^T D h, D = forward differences between neighbouring box cells along
    each axis (none across the faces), written with np.diff."""
    out = np.zeros_like(h)
    for ax in range(3):
        d = np.diff(h, axis=ax)
        z = np.zeros_like(np.take(h, [0], axis=ax))
        out += np.concatenate([z, d], axis=ax) - np.concatenate([d, z], axis=ax)
    return out


def test_grad_energy_is_the_sum_of_squared_differences():
    h = random_volume(9, 151)
    want = sum(float((np.diff(h, axis=ax) ** 2).sum()) for ax in range(3))
    assert abs(o.grad_energy(h) - want) < 1e-12 * want
    assert abs(float((h * neumann_dtd(h)).sum()) - want) < 1e-12 * want


@pytest.mark.parametrize("n", [4, 5])
def test_prox_grad_is_the_dense_solve(n):
    """(I + a D^T D)^{-1} f solved densely (D^T D assembled column by column
    from the difference definition) against the DCT-diagonalised oracle."""
    M = dense(neumann_dtd, n**3, (n, n, n))
    f = random_volume(n, 152 + n)
    for a in (0.0, 0.3, 17.0):
        want = np.linalg.solve(np.eye(n**3) + a * M, f.ravel()).reshape(f.shape)
        got = o.prox_grad(f, a)
        assert np.max(np.abs(got - want)) < 1e-12 * np.abs(f).max()


def test_prox_grad_on_cosine_modes():
    """The separable cosine modes cos(pi k (2i + 1) / (2n)) are eigenvectors of
    the zero-flux D^T D with eigenvalue sum_axes 4 sin^2(pi k / (2n)), so the
    prox divides them by 1 + a mu (closed form), on grids larger than the dense
    check reaches, ragged and even."""
    for n, a in ((13, 0.7), (24, 5.0)):
        i = np.arange(n)
        for kz, ky, kx in ((0, 0, 1), (1, 2, 3), (n - 1, 5, 0), (4, n - 2, n - 1)):
            fz, fy, fx = (np.cos(np.pi * k * (2 * i + 1) / (2 * n)) for k in (kz, ky, kx))
            f = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
            mu = sum(4 * np.sin(np.pi * k / (2 * n)) ** 2 for k in (kz, ky, kx))
            got = o.prox_grad(f, a)
            assert np.max(np.abs(got - f / (1 + a * mu))) < 1e-12


def test_prox_grad_optimality_and_kernel():
    """The prox satisfies h - f + a D^T D h = 0 (first-order optimality of
    1/2 ||h - f||^2 + a/2 ||D h||^2) on a ragged grid, and leaves constants,
    the kernel of D, unchanged."""
    n, a = 13, 3.7
    f = random_volume(n, 155)
    h = o.prox_grad(f, a)
    assert np.linalg.norm(h - f + a * neumann_dtd(h)) < 1e-12 * np.linalg.norm(f)
    const = np.full((n, n, n), 2.5)
    assert np.max(np.abs(o.prox_grad(const, a) - const)) < 1e-13
    assert np.max(np.abs(o.prox_grad(f, 0.0) - f)) < 1e-13


def test_fb_gradient_regulariser_first_step_and_objective():
    """From h_0 = 0 one step with R = 1/2 |grad h|^2 is prox(s A^T g) with
    a = s lambda / dx^2; the first objective is 1/2 ||g||^2 (R(0) = 0) and the
    second carries lambda R(h_1) = lambda/2 ||D h_1||^2 / dx^2."""
    n, nth, T, s, lam = 10, 6, 0.5, 0.05, 0.3
    c = random_speed(n, 157)
    g = random_data(nth, n, 158)
    dx = 2.0 / n
    h1, st1, _ = o.fb_masked(c, g, T, lam, s, 1, reg=1)
    want = o.prox_grad(s * o.adjoint(c, g, T), s * lam / dx**2)
    assert np.max(np.abs(h1 - want)) < 1e-13 * np.abs(want).max()
    assert abs(st1[0, 0] - 0.5 * float((g * g).sum())) < 1e-12 * st1[0, 0]
    h2, st2, _ = o.fb_masked(c, g, T, lam, s, 2, reg=1)
    r = o.forward(c, h1, T, nth) - g
    obj = 0.5 * float((r * r).sum()) + lam * 0.5 * o.grad_energy(h1) / dx**2
    assert abs(st2[1, 0] - obj) < 1e-12 * obj
    with pytest.raises(ValueError):
        o.fb_masked(c, g, T, lam, s, 1, reg=1, support=np.ones((n, n, n)))


def test_fb_gradient_regulariser_stationary_point():
    """At the fixed point of FB with R = 1/2 |grad h|^2 the gradient of the
    smooth functional vanishes: A^T (A h - g) + lambda D^T D h / dx^2 = 0."""
    n, nth, T, lam = 6, 6, 0.5, 0.02
    c = random_speed(n, 159)
    g = random_data(nth, n, 160)
    dx = 2.0 / n
    L = o.power(c, random_volume(n, 161), T, nth, iters=200)
    h, st, k = o.fb_masked(c, g, T, lam, 1.0 / L, 3000, reg=1)
    grad = o.adjoint(c, o.forward(c, h, T, nth) - g, T) + lam * neumann_dtd(h) / dx**2
    assert np.linalg.norm(grad) < 1e-8 * np.linalg.norm(o.adjoint(c, g, T))
    assert np.all(np.diff(st[:, 0]) <= 1e-12 * st[0, 0])  # monotone objective (s = 1/L)


def test_two_step_gradient_regulariser_first_iterate():
    """Algorithm 9 with R = 1/2 |grad h|^2: h_1 = prox(s W^T X^{-1} G)."""
    n, nth, T, s, lam = 10, 8, 0.5, 0.4, 0.2
    c = random_speed(n, 163)
    G = random_data(nth, n, 164)
    dx = 2.0 / n
    h1, _, _ = o.fb_two_step(c, G, T, lam, s, 1, reg=1)
    want = o.prox_grad(s * o.wave_pad(c, o.fbp(G), T, 0, transpose=True), s * lam / dx**2)
    assert np.max(np.abs(h1 - want)) < 1e-13 * np.abs(want).max()
