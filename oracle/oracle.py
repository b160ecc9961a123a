"""ctypes binding of the plain FP64 CPU oracle (``oracle/ffpat_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` use it; the product library never does.

Every wrapper takes and returns float64 NumPy arrays in ``[z][y][x]`` (volumes)
or ``[theta][z][xi]`` (projection data) layout.  The citations are to
Haltmeier, Zangerl, Nuster, Nguyen (2019): wave model eq. (1)-(3), the X-ray
transform eq. (4), the preconditioner / backprojection / adjoint of Sec. 3.1,
and Algorithm 8 with its proximal map (Sec. 3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffpat_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libffpat_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over planes)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.ffo_time_steps.restype = ctypes.c_int
            L.ffo_time_steps.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _D]
            L.ffo_kappa.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
            L.ffo_max.restype = ctypes.c_double
            L.ffo_max.argtypes = [ctypes.c_size_t, _D]
            L.ffo_wave.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.ffo_wave_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.ffo_angles.argtypes = [ctypes.c_int, _D, _D]
            L.ffo_ray_samples.restype = ctypes.c_int
            L.ffo_ray_samples.argtypes = [ctypes.c_int]
            L.ffo_sample_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32, _I32, _D]
            L.ffo_sample_points_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _I32, _I32, _D]
            L.ffo_project.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_project_rays.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _I32, _D]
            L.ffo_backproject.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_ramp_tap.restype = ctypes.c_double
            L.ffo_ramp_tap.argtypes = [ctypes.c_int, ctypes.c_int]
            L.ffo_ramp.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_forward.restype = ctypes.c_int
            L.ffo_forward.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _D, _D, _D]
            L.ffo_adjoint.restype = ctypes.c_int
            L.ffo_adjoint.argtypes = L.ffo_forward.argtypes
            L.ffo_forward_pad.restype = ctypes.c_int
            L.ffo_forward_pad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _D, _D, _D]
            L.ffo_adjoint_pad.restype = ctypes.c_int
            L.ffo_adjoint_pad.argtypes = L.ffo_forward_pad.argtypes
            L.ffo_wave_pad.restype = ctypes.c_int
            L.ffo_wave_pad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _D, _D, _D, ctypes.c_int]
            L.ffo_project_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_backproject_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_ramp_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_fbp_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_power_ex.restype = ctypes.c_double
            L.ffo_power_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                       ctypes.c_int]
            L.ffo_power.restype = ctypes.c_double
            L.ffo_power.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, _D, _D, ctypes.c_int]
            L.ffo_fb.restype = ctypes.c_int
            L.ffo_fb.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_double, _D, _D]
            L.ffo_grad.restype = ctypes.c_int
            L.ffo_grad.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   _D, _D, _D, _D, _D]
            L.ffo_fbp.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
            L.ffo_fb_two_step.restype = ctypes.c_int
            L.ffo_fb_two_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _D, _D, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_double, _D, _D]
            L.ffo_grad_energy.restype = ctypes.c_double
            L.ffo_grad_energy.argtypes = [ctypes.c_int, _D]
            L.ffo_prox_grad.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
            L.ffo_fb_ex.restype = ctypes.c_int
            L.ffo_fb_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_int,
                                    ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double, _D, _D]
            L.ffo_num_threads.restype = ctypes.c_int
            L.ffo_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().ffo_num_threads()


def set_num_threads(k: int) -> None:
    lib().ffo_set_num_threads(int(k))


def time_steps(n: int, T: float, cfl: float, cmax: float):
    """(Nt, dt) of the leapfrog discretisation of eq. (1) up to time T."""
    dt = ctypes.c_double()
    nt = lib().ffo_time_steps(n, T, cfl, cmax, ctypes.byref(dt))
    return nt, dt.value


def kappa(n: int, dt: float, c) -> np.ndarray:
    c = _f64(c)
    out = np.empty_like(c)
    lib().ffo_kappa(n, dt, _p(c), _p(out))
    return out


def wave(kap, h, nt: int) -> np.ndarray:
    """W_T h for an explicit step count nt (kappa already holds dt)."""
    kap, h = _f64(kap), _f64(h)
    out = np.empty_like(h)
    lib().ffo_wave(h.shape[0], int(nt), _p(kap), _p(h), _p(out))
    return out


def wave_adjoint(kap, g, nt: int) -> np.ndarray:
    kap, g = _f64(kap), _f64(g)
    out = np.empty_like(g)
    lib().ffo_wave_adjoint(g.shape[0], int(nt), _p(kap), _p(g), _p(out))
    return out


def angles(nth: int):
    cs = np.empty(nth)
    sn = np.empty(nth)
    lib().ffo_angles(nth, _p(cs), _p(sn))
    return cs, sn


def ray_samples(n: int) -> int:
    return lib().ffo_ray_samples(n)


def sample_points(n: int, nth: int, jkm, nimg: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """(i0, j0) corners and (fx, fy) fractions of the ray samples (j, k, m) on
    a data grid of n cells of size 2 / nimg (default n)."""
    jkm = np.ascontiguousarray(jkm, dtype=np.int32).reshape(-1, 3)
    ij = np.empty((jkm.shape[0], 2), dtype=np.int32)
    f = np.empty((jkm.shape[0], 2), dtype=np.float64)
    lib().ffo_sample_points_g(n, nimg or n, nth, jkm.shape[0], jkm.ctypes.data_as(_I32),
                              ij.ctypes.data_as(_I32), _p(f))
    return ij, f


def project(p, nth: int, nimg: int | None = None) -> np.ndarray:
    """P of the planes of p (ng^3); the cells have size 2 / nimg (default ng:
    the box [-1, 1]^3; nimg < ng: a wave grid padded around the box)."""
    p = _f64(p)
    n = p.shape[0]
    g = np.empty((nth, n, n))
    lib().ffo_project_g(n, nimg or n, nth, _p(p), _p(g))
    return g


def project_rays(p, nth: int, jlk) -> np.ndarray:
    """g[j][l][k] of project() for the listed (j, l, k) only."""
    p = _f64(p)
    jlk = np.ascontiguousarray(jlk, dtype=np.int32).reshape(-1, 3)
    out = np.empty(jlk.shape[0])
    lib().ffo_project_rays(p.shape[0], nth, _p(p), jlk.shape[0], jlk.ctypes.data_as(_I32), _p(out))
    return out


def backproject(g, n: int, nimg: int | None = None) -> np.ndarray:
    g = _f64(g)
    out = np.empty((n, n, n))
    lib().ffo_backproject_g(n, nimg or n, g.shape[0], _p(g), _p(out))
    return out


def ramp_tap(n: int, d: int) -> float:
    return lib().ffo_ramp_tap(n, d)


def ramp(r, nimg: int | None = None) -> np.ndarray:
    r = _f64(r)
    out = np.empty_like(r)
    lib().ffo_ramp_g(r.shape[1], nimg or r.shape[1], r.shape[0], _p(r), _p(out))
    return out


def _image_n(c, pad: int) -> int:
    n = c.shape[0] - 2 * int(pad)
    if n < 1 or pad < 0:
        raise ValueError(f"c of side {c.shape[0]} cannot hold an image box padded by {pad}")
    return n


def forward(c, h, T: float, nth: int, cfl: float = 0.3, pad: int = 0) -> np.ndarray:
    """g = P W_T h (Problem 1, full data).  pad > 0: the wave runs on the grid
    enlarged by pad cells per side (c given on that grid, h on the image box)
    and g holds the projections of that whole grid, n_angles x nw x nw."""
    c, h = _f64(c), _f64(h)
    n = h.shape[0]
    assert _image_n(c, pad) == n
    nw = n + 2 * pad
    g = np.empty((nth, nw, nw))
    lib().ffo_forward_pad(n, pad, T, cfl, nth, _p(c), _p(h), _p(g))
    return g


def adjoint(c, g, T: float, cfl: float = 0.3, pad: int = 0) -> np.ndarray:
    """h = W_T^T P^T g."""
    c, g = _f64(c), _f64(g)
    n = _image_n(c, pad)
    h = np.empty((n, n, n))
    lib().ffo_adjoint_pad(n, pad, T, cfl, g.shape[0], _p(c), _p(g), _p(h))
    return h


def wave_pad(c, u, T: float, pad: int, transpose: bool = False, cfl: float = 0.3) -> np.ndarray:
    """W_T E (box source u -> field on the wave grid padded by pad cells), or
    its transpose E^T W_T^T (wave-grid volume u -> box)."""
    c, u = _f64(c), _f64(u)
    n = _image_n(c, pad)
    m = n if transpose else n + 2 * pad
    out = np.empty((m, m, m))
    lib().ffo_wave_pad(n, pad, T, cfl, _p(c), _p(u), _p(out), int(bool(transpose)))
    return out


def power(c, v0, T: float, nth: int, precond: int = 0, iters: int = 20, cfl: float = 0.3,
          pad: int = 0, mask=None) -> float:
    """Largest eigenvalue of A^T chi Lambda chi A by power iteration from v0."""
    c, v0 = _f64(c), _f64(v0)
    m = _f64(mask) if mask is not None else None
    return lib().ffo_power_ex(_image_n(c, pad), pad, T, cfl, nth, precond, _p(c),
                              _p(m) if m is not None else None, _p(v0), iters)


def fb(c, g, T: float, lam: float, step: float, iters: int, h0=None, precond: int = 0,
       tol: float = 0.0, cfl: float = 0.3):
    """Algorithm 8 with R = l1 + positivity.  Returns (h, stats[k, 4], iters_done)."""
    c, g = _f64(c), _f64(g)
    n = c.shape[0]
    h = np.zeros((n, n, n)) if h0 is None else _f64(h0).copy()
    stats = np.zeros((max(iters, 1), 4))
    k = lib().ffo_fb(n, T, cfl, g.shape[0], precond, _p(c), _p(g), lam, step, iters, tol,
                     _p(h), _p(stats))
    return h, stats[:k], k


def grad(c, h, grad_g, T: float, cfl: float = 0.3):
    """(d/dh, d/dc) of <grad_g, A(c) h>, with dt held at its value for c."""
    c, h, grad_g = _f64(c), _f64(h), _f64(grad_g)
    n = c.shape[0]
    gh = np.empty((n, n, n))
    gc = np.empty((n, n, n))
    lib().ffo_grad(n, T, cfl, grad_g.shape[0], _p(c), _p(h), _p(grad_g), _p(gh), _p(gc))
    return gh, gc


def fbp(G, nimg: int | None = None) -> np.ndarray:
    """X^{-1} G = (2 pi / (n_angles dx)) P^T Lambda G, plane by plane (cells
    of size dx = 2 / nimg, default the grid size of G)."""
    G = _f64(G)
    n = G.shape[1]
    out = np.empty((n, n, n))
    lib().ffo_fbp_g(n, nimg or n, G.shape[0], _p(G), _p(out))
    return out


def fb_two_step(c, G, T: float, lam: float, step: float, iters: int, h0=None, tol: float = 0.0,
                cfl: float = 0.3, pad: int = 0, reg: int = 0):
    """Algorithm 9 with R = l1 + positivity (reg 0) or 1/2 |grad h|^2 (reg 1).
    Returns (h, stats[k, 4], iters_done)."""
    c, G = _f64(c), _f64(G)
    n = _image_n(c, pad)
    h = np.zeros((n, n, n)) if h0 is None else _f64(h0).copy()
    stats = np.zeros((max(iters, 1), 4))
    k = lib().ffo_fb_two_step(n, pad, T, cfl, G.shape[0], _p(c), _p(G), int(reg), lam, step,
                              iters, tol, _p(h), _p(stats))
    return h, stats[:k], k


def fb_masked(c, g, T: float, lam: float, step: float, iters: int, mask=None, support=None,
              h0=None, precond: int = 0, tol: float = 0.0, cfl: float = 0.3, pad: int = 0,
              reg: int = 0):
    """Algorithm 8 with the data mask chi_M (Problem 1) and the source support
    chi_V: r = A^T chi Lambda chi (A h - g), h+ = chi_V max(h - s r - s lambda, 0).
    pad > 0: the wave on the grid padded by pad cells (c on that grid).
    reg = 1: R = 1/2 |grad h|^2 (prox_grad) instead of l1 + positivity."""
    c, g = _f64(c), _f64(g)
    n = _image_n(c, pad)
    h = np.zeros((n, n, n)) if h0 is None else _f64(h0).copy()
    stats = np.zeros((max(iters, 1), 4))
    m = _f64(mask) if mask is not None else None
    sp = _f64(support) if support is not None else None
    k = lib().ffo_fb_ex(n, pad, T, cfl, g.shape[0], precond, _p(c), _p(g),
                        _p(m) if m is not None else None, _p(sp) if sp is not None else None,
                        int(reg), lam, step, iters, tol, _p(h), _p(stats))
    if k < 0:
        raise ValueError("the gradient regulariser takes no support mask")
    return h, stats[:k], k


def grad_energy(h) -> float:
    """<D h, D h>: squared forward differences between neighbouring box cells."""
    h = _f64(h)
    return lib().ffo_grad_energy(h.shape[0], _p(h))


def prox_grad(f, a: float) -> np.ndarray:
    """(I + a D^T D)^{-1} f: the prox of s lambda R, R = 1/2 |grad h|^2, a = s lambda / dx^2
    (Sec. 3.2 proximal map, Sec. 5 regulariser), by conjugate gradients on the
    difference definition of D^T D."""
    f = _f64(f)
    out = np.empty_like(f)
    lib().ffo_prox_grad(f.shape[0], float(a), _p(f), _p(out))
    return out
