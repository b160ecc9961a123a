"""The stored oracle values of tests/golden/oracle_n8.txt (8^3, 6 angles:
A h, A^T g and two iterations of Algorithm 8).  On the CPU the oracle must
still reproduce them (a change of its arithmetic shows up here and must come
with a regenerated file); on the GPU the CUDA path is compared with the stored
values, without running the oracle."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden as G  # noqa: E402

from tolerances import tol  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_oracle_reproduces_the_stored_values():
    want = G.load()
    got = G.compute()
    for k in want:
        assert got[k].shape == want[k].shape
        assert _rel(got[k], want[k]) < 1e-13, k


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_gpu_matches_the_stored_values(prec):
    torch = pytest.importorskip("torch")
    from paper_1901_06503_gb300 import build_lib
    from paper_1901_06503_gb300 import ffpat as F
    from paper_1901_06503_gb300.inputs import add_noise
    build_lib.build()
    want = G.load()
    c, h, noise = G.case()
    prob = F.problem(G.N, G.T, G.NTH, prec)
    dt = F.torch_dtype(prob)
    if prec != F.FP64:  # FP32 problems take FP32 inputs; the stored values are FP64
        c, h = c.astype(np.float32).astype(np.float64), h.astype(np.float32).astype(np.float64)
    cd = torch.as_tensor(c, device="cuda").to(dt)
    g = F.forward(prob, cd, torch.as_tensor(h, device="cuda").to(dt))
    assert _rel(g.double().cpu().numpy(), want["A_h"]) < tol(prec)
    gd = torch.as_tensor(add_noise(want["A_h"], noise, 0.01), device="cuda").to(dt)
    a = F.adjoint(prob, cd, gd)
    assert _rel(a.double().cpu().numpy(), want["At_g"]) < tol(prec)
    hk, _, _ = F.fb_solve(prob, cd, gd, G.LAM, G.STEP, G.ITERS, history=False)
    torch.cuda.synchronize()
    assert _rel(hk.double().cpu().numpy(), want["fb_h2"]) < tol(prec)
