"""Host-side tests of the C ABI: the library builds for sm_103a, loads, exports
every symbol the header declares, and its host-only logic (time discretisation,
angle tables, argument validation) agrees with the oracle.  No kernel runs."""
import ctypes

import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F


@pytest.fixture(scope="module")
def L():
    build_lib.build()
    return F.lib()


def test_exports_every_declared_symbol(L):
    syms = F.header_symbols()
    assert "ffpat_forward" in syms and "ffpat_fb_solve" in syms and len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s


def test_problem_info_matches_oracle(L):
    for n, T, cmax in [(32, 1.0, 1.2), (128, 1.2, 1.3), (384, 1.5, 1.4), (48, 0.37, 1.173),
                       (16, 1e-6, 1.0)]:
        prob = F.problem(n, T, 8)
        nt, dt, ns = F.problem_info(prob, cmax)
        ont, odt = o.time_steps(n, T, 0.3, cmax)
        assert (nt, dt) == (ont, odt)
        assert ns == o.ray_samples(n)


def test_angle_table_bit_exact(L):
    for nth in (1, 6, 24, 90, 180, 1000):
        tab = F.debug_tables(F.problem(16, 1.0, nth))
        cs, sn = o.angles(nth)
        assert np.array_equal(tab[:, 0], cs) and np.array_equal(tab[:, 1], sn)


def test_workspace_grows_with_problem(L):
    small = F.workspace_bytes(F.problem(32, 1.0, 24))
    big = F.workspace_bytes(F.problem(64, 1.0, 24))
    kahan = F.workspace_bytes(F.problem(64, 1.0, 24, F.FP32_KAHAN))
    fp32 = F.workspace_bytes(F.problem(64, 1.0, 24, F.FP32))
    assert big > small > 0 and kahan > fp32
    # FP64 stores 8-byte values: at least kappa + 2 states + 2 scratch volumes
    assert big >= 5 * 64**3 * 8
    # padding: kappa, two states and the input on the wave grid on top
    padded = F.workspace_bytes(F.problem(64, 1.0, 24, pad=32))
    assert padded >= big + 4 * (128**3 - 64**3) * 8


def test_padding_rejected_where_unsupported(L):
    prob = F.problem(16, 1.0, 4, F.FP32_KAHAN, pad=4)
    assert L.ffpat_ckpt_bytes(ctypes.byref(prob), 10, 4) == 0
    assert b"pad" in L.ffpat_last_error()


@pytest.mark.parametrize("bad", [
    dict(n=0), dict(n=5000), dict(T=0.0), dict(T=float("nan")), dict(cfl=0.51), dict(cfl=0.0),
    dict(n_angles=0), dict(precision=7), dict(precond=3), dict(pad=-1), dict(pad=2049),
    dict(n=2048, pad=1025)])
def test_invalid_problems_rejected(L, bad):
    kw = dict(n=16, T=1.0, n_angles=4, precision=0, precond=0, cfl=0.3, pad=0)
    kw.update(bad)
    prob = F.Problem(kw["n"], kw["T"], kw["cfl"], kw["n_angles"], kw["precision"], kw["precond"],
                     kw["pad"])
    assert L.ffpat_workspace_bytes(ctypes.byref(prob)) == 0
    assert L.ffpat_last_error()
    # entry points reject the problem before touching the GPU
    rc = L.ffpat_forward(ctypes.byref(prob), None, None, None, None, 0, None)
    assert rc == F.EINVAL


def test_missing_workspace_rejected(L):
    prob = F.problem(16, 1.0, 4)
    rc = L.ffpat_forward(ctypes.byref(prob), None, None, None, None, 0, None)
    assert rc == F.EINVAL and b"workspace" in L.ffpat_last_error()
    ws = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    rc = L.ffpat_fb_solve(ctypes.byref(prob), None, None, 0.0, 1.0, 1, 0.0, None, None, None,
                          ws, 1024, None)
    assert rc == F.ENOMEM


def test_problem_info_rejects_bad_speed(L):
    with pytest.raises(F.FFPATError):
        F.problem_info(F.problem(16, 1.0, 4), 0.0)


def test_stencil_path_range(L):
    """Paths 0 (automatic) to 4 (resident time loop) are accepted without a
    GPU; anything else is rejected with a message."""
    try:
        for path in range(5):
            assert L.ffpat_set_stencil_path(path) == 0
        for bad in (-1, 5):
            assert L.ffpat_set_stencil_path(bad) == F.EINVAL
            assert b"stencil path" in L.ffpat_last_error()
    finally:
        L.ffpat_set_stencil_path(0)


def test_fma_rate_probe_rejects_bad_arguments(L):
    out = ctypes.c_double(0.0)
    assert L.ffpat_debug_fma_rate(3, ctypes.byref(out), None) == F.EINVAL
    assert L.ffpat_debug_fma_rate(0, None, None) == F.EINVAL
