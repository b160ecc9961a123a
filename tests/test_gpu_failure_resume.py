"""Failure detection without a GPU fault, and resume of Algorithm 8.

* A kernel waits on an mbarrier that nothing completes; its bounded wait runs
  out, the device status word reads FFPAT_ETIMEDOUT on the host, and the
  context stays usable (a forward pass afterwards still matches the oracle).
  While the word is set, the stencil kernels skip their work, so the status is
  cleared before continuing.
* FB keeps no state besides the iterate: k1 + k2 iterations split over two
  calls (warm start from the saved h) equal k1 + k2 iterations in one call,
  bit for bit.
"""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import add_noise, config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    F.lib()


def test_bounded_wait_timeout_is_reported_and_recoverable():
    assert F.device_status(clear=True) == 0
    F.debug_wait_timeout(20000)  # 20 ms bound
    assert F.device_status() == F.ETIMEDOUT
    assert F.device_status(clear=True) == F.ETIMEDOUT
    assert F.device_status() == 0
    w = config(1)
    prob = F.problem(w.n, w.T, w.n_angles, F.FP32_KAHAN)
    g = F.forward(prob, torch.as_tensor(w.c, device="cuda").float(),
                  torch.as_tensor(w.h, device="cuda").float())
    torch.cuda.synchronize()
    want = o.forward(w.c.astype(np.float32).astype(np.float64),
                     w.h.astype(np.float32).astype(np.float64), w.T, w.n_angles)
    assert np.linalg.norm(g.double().cpu().numpy() - want) / np.linalg.norm(want) < 2e-5


@pytest.mark.parametrize("prec", [F.FP64, F.FP32_KAHAN])
def test_resume_is_bit_identical(prec):
    w = config(1)
    prob = F.problem(w.n, w.T, w.n_angles, prec)
    dt = F.torch_dtype(prob)
    c = torch.as_tensor(w.c, device="cuda").to(dt)
    g = torch.as_tensor(add_noise(o.forward(w.c, w.h, w.T, w.n_angles), w.noise, w.noise_rel),
                        device="cuda").to(dt)
    h_all, _, _ = F.fb_solve(prob, c, g, w.lam, 0.05, 7)
    h_part, _, _ = F.fb_solve(prob, c, g, w.lam, 0.05, 3)
    saved = h_part.cpu().clone()  # checkpoint of the iterate
    h_res, st, _ = F.fb_solve(prob, c, g, w.lam, 0.05, 4, h=saved.to("cuda"))
    torch.cuda.synchronize()
    assert st["iters_done"] == 4
    assert torch.equal(h_res, h_all)
