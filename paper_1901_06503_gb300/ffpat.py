"""Thin ctypes binding of the C ABI in ``include/ffpat.h`` (libffpat.so).

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: a missing or unloadable library
raises.

Names follow the ABI (``ffpat_forward`` -> :func:`forward`, ...).  Volumes are
``[z][y][x]`` tensors of shape (N, N, N); projection data are
``[theta][z][xi]`` tensors of shape (n_angles, N, N); float64 for FFPAT_FP64
problems, float32 otherwise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FFPAT_LIB=<path> loads another build of the same library (e.g. the sanitizer build)
LIB_PATH = os.environ.get("FFPAT_LIB") or os.path.join(HERE, "libffpat.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ffpat.h")

FP64, FP32, FP32_KAHAN = 0, 1, 2
PRECOND_NONE, PRECOND_RAMP = 0, 1
REG_L1_POS, REG_GRAD2 = 0, 1
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEDOUT, ECANCELED, PENDING = 0, -1, -2, -3, -4, -5, -6, 1
PRECISION_NAMES = {FP64: "fp64", FP32: "fp32", FP32_KAHAN: "fp32-kahan"}


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("T", ctypes.c_double), ("cfl", ctypes.c_double),
                ("n_angles", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def __repr__(self):
        return (f"Problem(n={self.n}, T={self.T}, cfl={self.cfl}, n_angles={self.n_angles}, "
                f"precision={PRECISION_NAMES.get(self.precision, self.precision)}, "
                f"precond={self.precond}, pad={self.pad})")


class FBStats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("objective", ctypes.c_double),
                ("resid_norm", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("step", ctypes.c_double), ("opnorm_sq", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_int64), ("step_ms", ctypes.c_double),
                ("step_bytes", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("steps", ctypes.c_int64)]


class ServingStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("point_steps", ctypes.c_double),
                ("ticks", ctypes.c_int64), ("active", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("hbm_in_use", ctypes.c_size_t)]


class FFPATError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ffpat error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_PR = ctypes.POINTER(Problem)


def _declare(L):
    i32, i64, f64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ffpat_last_error": (ctypes.c_char_p, []),
        "ffpat_version": (ctypes.c_char_p, []),
        "ffpat_workspace_bytes": (sz, [_PR]),
        "ffpat_problem_info": (ctypes.c_int, [_PR, f64, ctypes.POINTER(i32), ctypes.POINTER(f64),
                                              ctypes.POINTER(i32)]),
        "ffpat_debug_tables": (ctypes.c_int, [_PR, _P]),
        "ffpat_debug_samples": (ctypes.c_int, [_PR, i32, _P, _P, _P, _P]),
        "ffpat_forward": (ctypes.c_int, [_PR, _P, _P, _P, _P, sz, _P]),
        "ffpat_adjoint": (ctypes.c_int, [_PR, _P, _P, _P, _P, sz, _P]),
        "ffpat_wave": (ctypes.c_int, [_PR, _P, _P, _P, i32, _P, sz, _P]),
        "ffpat_project": (ctypes.c_int, [_PR, _P, _P, _P]),
        "ffpat_backproject": (ctypes.c_int, [_PR, _P, _P, _P]),
        "ffpat_ramp": (ctypes.c_int, [_PR, _P, _P, _P]),
        "ffpat_opnorm": (ctypes.c_int, [_PR, _P, _P, i32, ctypes.POINTER(f64), _P, sz, _P]),
        "ffpat_fb_solve": (ctypes.c_int, [_PR, _P, _P, f64, f64, i32, f64, _P,
                                          ctypes.POINTER(FBStats), _P, _P, sz, _P]),
        "ffpat_fbp": (ctypes.c_int, [_PR, _P, _P, _P, sz, _P]),
        "ffpat_fb_solve_ex": (ctypes.c_int, [_PR, _P, _P, _P, _P, i32, f64, f64, i32, f64, _P,
                                             ctypes.POINTER(FBStats), _P, _P, sz, _P]),
        "ffpat_fb_two_step_ex": (ctypes.c_int, [_PR, _P, _P, i32, f64, f64, i32, f64, _P,
                                                ctypes.POINTER(FBStats), _P, _P, sz, _P]),
        "ffpat_prox_grad": (ctypes.c_int, [_PR, f64, _P, _P, _P, sz, _P]),
        "ffpat_fb_two_step": (ctypes.c_int, [_PR, _P, _P, f64, f64, i32, f64, _P,
                                             ctypes.POINTER(FBStats), _P, _P, sz, _P]),
        "ffpat_profile_enable": (ctypes.c_int, [i32]),
        "ffpat_profile_read": (ctypes.c_int, [ctypes.POINTER(Profile)]),
        "ffpat_launch_count": (i64, []),
        "ffpat_set_stencil_path": (ctypes.c_int, [i32]),
        "ffpat_device_status": (ctypes.c_int, [i32]),
        "ffpat_debug_wait_timeout": (ctypes.c_int, [i32, _P]),
        "ffpat_debug_fma_rate": (ctypes.c_int, [i32, ctypes.POINTER(f64), _P]),
        "ffpat_forward_noalloc": (ctypes.c_int, [_PR, _P, _P, _P, _P]),
        "ffpat_ckpt_bytes": (sz, [_PR, i32, i32]),
        "ffpat_forward_ckpt": (ctypes.c_int, [_PR, _P, _P, _P, i32, _P, sz, _P, sz, _P]),
        "ffpat_backward": (ctypes.c_int, [_PR, _P, _P, _P, _P, i32, _P, sz, _P, sz, _P]),
        "ffpat_server_create": (ctypes.c_int, [sz, i32, ctypes.POINTER(ctypes.c_void_p)]),
        "ffpat_submit": (ctypes.c_int, [_P, _PR, _P, _P, f64, f64, i32,
                                        ctypes.POINTER(ctypes.c_uint64)]),
        "ffpat_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(FBStats)]),
        "ffpat_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
        "ffpat_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServingStats)]),
        "ffpat_server_destroy": (ctypes.c_int, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """Load libffpat.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FFPATError(ECUDA, f"{LIB_PATH} is missing: build it with "
                                        "paper_1901_06503_gb300.build_lib.build()")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Every function the public header declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ffpat_[a-z0-9_]+)\s*\(", text)))


def _check(rc):
    if rc < 0:
        raise FFPATError(rc, lib().ffpat_last_error().decode())
    return rc


def problem(n: int, T: float, n_angles: int, precision: int = FP64, precond: int = 0,
            cfl: float = 0.3, pad: int = 0) -> Problem:
    """pad > 0: the wave runs on the grid of n + 2 pad points per axis (c is
    given there); sources, images and data stay on the n^3 box."""
    return Problem(int(n), float(T), float(cfl), int(n_angles), int(precision), int(precond),
                   int(pad))


def torch_dtype(prob: Problem):
    import torch
    return torch.float64 if prob.precision == FP64 else torch.float32


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, prob, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch_dtype(prob):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {torch_dtype(prob)}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def vol_shape(prob):
    return (prob.n, prob.n, prob.n)


def wave_shape(prob):
    """Shape of the sound speed: the wave grid, n + 2 pad points per axis."""
    nw = prob.n + 2 * prob.pad
    return (nw, nw, nw)


def data_shape(prob):
    """Projections of the wave grid: n_angles x nw x nw."""
    nw = prob.n + 2 * prob.pad
    return (prob.n_angles, nw, nw)


def workspace_bytes(prob: Problem) -> int:
    b = lib().ffpat_workspace_bytes(ctypes.byref(prob))
    if b == 0:
        raise FFPATError(EINVAL, lib().ffpat_last_error().decode())
    return int(b)


def workspace(prob: Problem, device="cuda"):
    import torch
    return torch.empty(workspace_bytes(prob), dtype=torch.uint8, device=device)


def _ws(prob, ws, device):
    if ws is None:
        ws = workspace(prob, device)
    return ws, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def _empty(prob, shape, like):
    import torch
    return torch.empty(shape, dtype=torch_dtype(prob), device=like.device)


def problem_info(prob: Problem, cmax: float):
    nt, dt, ns = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().ffpat_problem_info(ctypes.byref(prob), cmax, ctypes.byref(nt), ctypes.byref(dt),
                                    ctypes.byref(ns)))
    return nt.value, dt.value, ns.value


def debug_tables(prob: Problem) -> np.ndarray:
    out = np.empty((prob.n_angles, 2), dtype=np.float64)
    _check(lib().ffpat_debug_tables(ctypes.byref(prob), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def debug_samples(prob: Problem, jkm, device="cuda"):
    import torch
    jkm = torch.as_tensor(np.ascontiguousarray(jkm, dtype=np.int32).reshape(-1, 3), device=device)
    ij = torch.empty((jkm.shape[0], 2), dtype=torch.int32, device=device)
    f = torch.empty((jkm.shape[0], 2), dtype=torch.float64, device=device)
    _check(lib().ffpat_debug_samples(ctypes.byref(prob), jkm.shape[0], _P(jkm.data_ptr()),
                                     _P(ij.data_ptr()), _P(f.data_ptr()), _stream(None)))
    return ij.cpu().numpy(), f.cpu().numpy()


def forward(prob, c, h, g=None, ws=None, stream=None):
    """g = P W h."""
    g = _empty(prob, data_shape(prob), h) if g is None else g
    ws, wp, wn = _ws(prob, ws, h.device)
    _check(lib().ffpat_forward(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                               _dev(h, prob, vol_shape(prob), "h"),
                               _dev(g, prob, data_shape(prob), "g"), wp, wn, _stream(stream)))
    return g


def forward_noalloc(prob, c, h, g, stream=None):
    """g = P W h through the entry point that allocates nothing (static
    device scratch; wave grid N + 2 pad <= 64 with <= 180 angles).  `g` must be
    preallocated."""
    _check(lib().ffpat_forward_noalloc(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                       _dev(h, prob, vol_shape(prob), "h"),
                                       _dev(g, prob, data_shape(prob), "g"), _stream(stream)))
    return g


def ckpt_bytes(prob, nt: int, every: int) -> int:
    b = lib().ffpat_ckpt_bytes(ctypes.byref(prob), int(nt), int(every))
    if b == 0:
        raise FFPATError(EINVAL, "invalid checkpoint request")
    return int(b)


def forward_ckpt(prob, c, h, every, ckpt, g=None, ws=None, stream=None):
    """g = P W h, saving wavefield checkpoints every `every` steps into ckpt."""
    g = _empty(prob, data_shape(prob), h) if g is None else g
    ws, wp, wn = _ws(prob, ws, h.device)
    _check(lib().ffpat_forward_ckpt(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                    _dev(h, prob, vol_shape(prob), "h"),
                                    _dev(g, prob, data_shape(prob), "g"), int(every),
                                    ctypes.c_void_p(ckpt.data_ptr()), ctypes.c_size_t(ckpt.numel()),
                                    wp, wn, _stream(stream)))
    return g


def backward(prob, c, grad_g, every, ckpt, want_h=True, want_c=True, ws=None, stream=None):
    """(grad_h, grad_c) of <grad_g, A(c) h> after forward_ckpt."""
    gh = _empty(prob, vol_shape(prob), grad_g) if want_h else None
    gc = _empty(prob, vol_shape(prob), grad_g) if want_c else None
    ws, wp, wn = _ws(prob, ws, grad_g.device)
    _check(lib().ffpat_backward(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                _dev(grad_g, prob, data_shape(prob), "grad_g"),
                                _dev(gh, prob, vol_shape(prob), "grad_h") if want_h else None,
                                _dev(gc, prob, vol_shape(prob), "grad_c") if want_c else None,
                                int(every), ctypes.c_void_p(ckpt.data_ptr()),
                                ctypes.c_size_t(ckpt.numel()), wp, wn, _stream(stream)))
    return gh, gc


def adjoint(prob, c, g, h=None, ws=None, stream=None):
    """h = W^T P^T g."""
    h = _empty(prob, vol_shape(prob), g) if h is None else h
    ws, wp, wn = _ws(prob, ws, g.device)
    _check(lib().ffpat_adjoint(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                               _dev(g, prob, data_shape(prob), "g"),
                               _dev(h, prob, vol_shape(prob), "h"), wp, wn, _stream(stream)))
    return h


def wave(prob, c, x, out=None, transpose=False, ws=None, stream=None):
    """W x (box source -> wave grid) or W^T x (wave grid -> box)."""
    ins, outs = (wave_shape(prob), vol_shape(prob)) if transpose else (vol_shape(prob),
                                                                        wave_shape(prob))
    out = _empty(prob, outs, x) if out is None else out
    ws, wp, wn = _ws(prob, ws, x.device)
    _check(lib().ffpat_wave(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                            _dev(x, prob, ins, "in"), _dev(out, prob, outs, "out"),
                            int(bool(transpose)), wp, wn, _stream(stream)))
    return out


def project(prob, p, g=None, stream=None):
    """P of the wave grid (the box when pad = 0)."""
    g = _empty(prob, data_shape(prob), p) if g is None else g
    _check(lib().ffpat_project(ctypes.byref(prob), _dev(p, prob, wave_shape(prob), "p"),
                               _dev(g, prob, data_shape(prob), "g"), _stream(stream)))
    return g


def backproject(prob, g, h=None, stream=None):
    h = _empty(prob, wave_shape(prob), g) if h is None else h
    _check(lib().ffpat_backproject(ctypes.byref(prob), _dev(g, prob, data_shape(prob), "g"),
                                   _dev(h, prob, wave_shape(prob), "h"), _stream(stream)))
    return h


def ramp(prob, r, out=None, stream=None):
    out = _empty(prob, data_shape(prob), r) if out is None else out
    _check(lib().ffpat_ramp(ctypes.byref(prob), _dev(r, prob, data_shape(prob), "r"),
                            _dev(out, prob, data_shape(prob), "out"), _stream(stream)))
    return out


def opnorm(prob, c, v0, iters=20, ws=None, stream=None) -> float:
    ws, wp, wn = _ws(prob, ws, v0.device)
    est = ctypes.c_double()
    _check(lib().ffpat_opnorm(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                              _dev(v0, prob, vol_shape(prob), "v0"), int(iters),
                              ctypes.byref(est), wp, wn, _stream(stream)))
    return est.value


def fb_solve(prob, c, g, lam, step, max_iters, h=None, tol=0.0, ws=None, stream=None,
             history=True):
    """Algorithm 8; returns (h, stats dict, history array [k, 4] or None)."""
    import torch
    h = torch.zeros(vol_shape(prob), dtype=torch_dtype(prob), device=g.device) if h is None else h
    ws, wp, wn = _ws(prob, ws, g.device)
    st = FBStats()
    hist = np.zeros((max(int(max_iters), 1), 4)) if history else None
    hp = hist.ctypes.data_as(ctypes.c_void_p) if history else None
    _check(lib().ffpat_fb_solve(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                _dev(g, prob, data_shape(prob), "g"), float(lam), float(step),
                                int(max_iters), float(tol), _dev(h, prob, vol_shape(prob), "h"),
                                ctypes.byref(st), hp, wp, wn, _stream(stream)))
    d = st.as_dict()
    return h, d, (hist[: d["iters_done"]] if history else None)


def fb_solve_masked(prob, c, g, lam, step, max_iters, mask=None, support=None, h=None, tol=0.0,
                    ws=None, stream=None, history=True, reg=0):
    """Algorithm 8 with the data mask chi_M (data-shaped 0/1) and the source
    support chi_V (volume 0/1); None = full data / whole grid.  reg = REG_GRAD2
    uses R = 1/2 |grad h|^2 instead of l1 + positivity."""
    import torch
    h = torch.zeros(vol_shape(prob), dtype=torch_dtype(prob), device=g.device) if h is None else h
    ws, wp, wn = _ws(prob, ws, g.device)
    st = FBStats()
    hist = np.zeros((max(int(max_iters), 1), 4)) if history else None
    hp = hist.ctypes.data_as(ctypes.c_void_p) if history else None
    mp = _dev(mask, prob, data_shape(prob), "mask") if mask is not None else None
    sp = _dev(support, prob, vol_shape(prob), "support") if support is not None else None
    _check(lib().ffpat_fb_solve_ex(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                   _dev(g, prob, data_shape(prob), "g"), mp, sp, int(reg),
                                   float(lam),
                                   float(step), int(max_iters), float(tol),
                                   _dev(h, prob, vol_shape(prob), "h"), ctypes.byref(st), hp, wp,
                                   wn, _stream(stream)))
    d = st.as_dict()
    return h, d, (hist[: d["iters_done"]] if history else None)


def prox_grad(prob, f, a, out=None, ws=None, stream=None):
    """(I + a D^T D)^{-1} f: the prox of s lambda R, R = 1/2 |grad h|^2, a = s lambda / dx^2."""
    out = _empty(prob, vol_shape(prob), f) if out is None else out
    ws, wp, wn = _ws(prob, ws, f.device)
    _check(lib().ffpat_prox_grad(ctypes.byref(prob), float(a), _dev(f, prob, vol_shape(prob), "f"),
                                 _dev(out, prob, vol_shape(prob), "out"), wp, wn, _stream(stream)))
    return out


def fbp(prob, G, out=None, ws=None, stream=None):
    """X^{-1} G plane by plane (filtered backprojection onto the wave grid)."""
    out = _empty(prob, wave_shape(prob), G) if out is None else out
    ws, wp, wn = _ws(prob, ws, G.device)
    _check(lib().ffpat_fbp(ctypes.byref(prob), _dev(G, prob, data_shape(prob), "G"),
                           _dev(out, prob, wave_shape(prob), "out"), wp, wn, _stream(stream)))
    return out


def fb_two_step(prob, c, G, lam, step, max_iters, h=None, tol=0.0, ws=None, stream=None,
                history=True, reg=0):
    """Algorithm 9; returns (h, stats dict, history array [k, 4] or None).
    reg = REG_GRAD2: R = 1/2 |grad h|^2 (the paper's experiments)."""
    import torch
    h = torch.zeros(vol_shape(prob), dtype=torch_dtype(prob), device=G.device) if h is None else h
    ws, wp, wn = _ws(prob, ws, G.device)
    st = FBStats()
    hist = np.zeros((max(int(max_iters), 1), 4)) if history else None
    hp = hist.ctypes.data_as(ctypes.c_void_p) if history else None
    _check(lib().ffpat_fb_two_step_ex(ctypes.byref(prob), _dev(c, prob, wave_shape(prob), "c"),
                                      _dev(G, prob, data_shape(prob), "G"), int(reg), float(lam),
                                      float(step), int(max_iters), float(tol),
                                      _dev(h, prob, vol_shape(prob), "h"), ctypes.byref(st), hp,
                                      wp, wn, _stream(stream)))
    d = st.as_dict()
    return h, d, (hist[: d["iters_done"]] if history else None)


def profile_enable(on: bool = True) -> None:
    _check(lib().ffpat_profile_enable(1 if on else 0))


def profile_read() -> dict:
    p = Profile()
    _check(lib().ffpat_profile_read(ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in p._fields_}


def launch_count() -> int:
    return int(lib().ffpat_launch_count())


def set_stencil_path(path: int) -> None:
    """0 automatic, 1 plain 2.5D kernel, 2 single-step TMA kernel, 3 two-step TMA kernel,
    4 resident time loop (one cooperative launch, FP32 and FP32-Kahan, N <= 128)."""
    _check(lib().ffpat_set_stencil_path(int(path)))


def device_status(clear: bool = False) -> int:
    """0, or the negative status of the first device-side failure."""
    return int(lib().ffpat_device_status(1 if clear else 0))


def debug_wait_timeout(microseconds: int = 20000, stream=None) -> None:
    """Run a bounded device wait that cannot complete (sets FFPAT_ETIMEDOUT)."""
    _check(lib().ffpat_debug_wait_timeout(int(microseconds), _stream(stream)))


FMA_FP64, FMA_FP32, FMA_FP32X2 = 0, 1, 2


def debug_fma_rate(kind: int, stream=None) -> float:
    """Measured fused multiply-add rate of one pipe in FLOP/s (kind 0 FP64,
    1 FP32, 2 packed two-lane FP32)."""
    out = ctypes.c_double(0.0)
    _check(lib().ffpat_debug_fma_rate(int(kind), ctypes.byref(out), _stream(stream)))
    return float(out.value)


def version() -> str:
    return lib().ffpat_version().decode()


class Server:
    """Continuous-batching reconstruction server (ffpat_server_* / ffpat_submit /
    ffpat_poll).  Requests carry HOST arrays (float32 c: N^3, g: n_angles N^2)
    and run Algorithm 8 with the FP32-Kahan wave kernels on the device that is
    current at creation; their leapfrog steps share batched launches."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8):
        h = ctypes.c_void_p()
        _check(lib().ffpat_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, prob: Problem, c, g, lam: float, step: float, iters: int) -> int:
        c = np.ascontiguousarray(c, dtype=np.float32)
        g = np.ascontiguousarray(g, dtype=np.float32)
        if c.shape != vol_shape(prob) or g.shape != data_shape(prob):
            raise ValueError("c / g shapes do not match the problem")
        t = ctypes.c_uint64()
        _check(lib().ffpat_submit(self._h, ctypes.byref(prob), c.ctypes.data_as(_P),
                                  g.ctypes.data_as(_P), float(lam), float(step), int(iters),
                                  ctypes.byref(t)))
        self._shapes[t.value] = vol_shape(prob)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (h, stats); raises FFPATError on failure."""
        out = np.empty(self._shapes[ticket], dtype=np.float32)
        st = FBStats()
        rc = lib().ffpat_poll(self._h, ctypes.c_uint64(ticket), out.ctypes.data_as(_P),
                              ctypes.byref(st))
        if rc == PENDING:
            return None
        self._shapes.pop(ticket, None)
        _check(rc)
        return out, st.as_dict()

    def wait(self, ticket: int, timeout: float = 600.0, interval: float = 1e-3):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise FFPATError(ETIMEDOUT, f"request {ticket} not done after {timeout} s")
            time.sleep(interval)

    def cancel(self, ticket: int) -> None:
        _check(lib().ffpat_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        st = ServingStats()
        _check(lib().ffpat_server_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self) -> None:
        if self._h:
            lib().ffpat_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
