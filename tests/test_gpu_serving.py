"""Serving (ffpat_server_*): continuous batching of Algorithm-8 solves.

Each served result must equal the same solve run through ffpat_fb_solve, and
be the same alone and in a mix of requests of different sizes (bit for bit:
the batched leapfrog launch runs the per-point arithmetic of the single-problem
kernel).  Admission respects the HBM budget; a cancelled request fails alone.
"""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.inputs import add_noise, config

from tolerances import FP32_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    F.lib()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def request(n, nth, T, seed, iters=3, noise=0.01):
    w = config(1, n=n, seed=seed)
    c32 = w.c.astype(np.float32)
    g = o.forward(c32.astype(np.float64), w.h, T, nth)
    g = add_noise(g, np.random.default_rng(seed).standard_normal(g.shape), noise)
    prob = F.problem(n, T, nth, F.FP32_KAHAN)
    return prob, c32, g.astype(np.float32), iters


def fb_direct(prob, c, g, lam, step, iters):
    h, st, _ = F.fb_solve(prob, torch.as_tensor(c, device="cuda"), torch.as_tensor(g, device="cuda"),
                          lam, step, iters, history=False)
    torch.cuda.synchronize()
    return h.cpu().numpy(), st


def test_served_equals_fb_solve():
    prob, c, g, iters = request(32, 12, 0.5, 5)
    with F.Server(1 << 30, 4) as srv:
        for step in (0.05, 0.0):  # explicit step, then the power-iteration step
            t = srv.submit(prob, c, g, 1e-3, step, iters)
            h, st = srv.wait(t)
            h_ref, st_ref = fb_direct(prob, c, g, 1e-3, step, iters)
            assert np.array_equal(h, h_ref)
            assert st["step"] == st_ref["step"]
            assert abs(st["objective"] - st_ref["objective"]) <= 1e-12 * abs(st_ref["objective"])


def test_alone_equals_in_mix():
    reqs = [request(32, 12, 0.5, 11), request(48, 9, 0.4, 12, iters=2),
            request(64, 16, 0.6, 13), request(40, 7, 0.3, 14, iters=4)]
    alone = []
    for prob, c, g, it in reqs:
        with F.Server(1 << 30, 1) as srv:
            alone.append(srv.wait(srv.submit(prob, c, g, 1e-3, 0.02, it))[0])
    with F.Server(1 << 30, 8) as srv:
        tickets = [srv.submit(prob, c, g, 1e-3, 0.02, it) for prob, c, g, it in reqs]
        mixed = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)
    assert st["completed"] == 4 and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_budget_admission_and_cancel():
    reqs = [request(32, 12, 0.5, 21 + i) for i in range(4)]
    need = F.workspace_bytes(reqs[0][0]) + 8 * 32**3 + 4 * 12 * 32**2 + 4096
    with F.Server(need + need // 2, 8) as srv:  # room for one request at a time
        tickets = [srv.submit(prob, c, g, 1e-3, 0.02, it) for prob, c, g, it in reqs]
        srv.cancel(tickets[1])
        done = {}
        for t in (tickets[0], tickets[2], tickets[3]):
            done[t] = srv.wait(t)[0]
            assert srv.stats()["hbm_in_use"] <= need + need // 2
        with pytest.raises(F.FFPATError) as e:
            srv.wait(tickets[1])
        assert e.value.code == F.ECANCELED
        st = srv.stats()
    assert st["completed"] == 3 and st["cancelled"] == 1
    for t, (prob, c, g, it) in zip((tickets[0], tickets[2], tickets[3]), (reqs[0], reqs[2], reqs[3])):
        assert np.array_equal(done[t], fb_direct(prob, c, g, 1e-3, 0.02, it)[0])


def test_served_vs_oracle():
    prob, c, g, iters = request(32, 12, 0.5, 31, iters=4)
    with F.Server(1 << 30, 2) as srv:
        h, _ = srv.wait(srv.submit(prob, c, g, 1e-3, 0.02, iters))
    h_or, _, _ = o.fb(c.astype(np.float64), g.astype(np.float64), 0.5, 1e-3, 0.02, iters)
    assert rel(h, h_or) < FP32_TOL


def test_served_mix_vs_oracle_up_to_96():
    """A mix served concurrently -- requests of the serving workload's sizes
    64^3 (45 angles) and 96^3 (90 angles) beside a 128^3 request -- each
    request of at most 96^3 against the oracle's Algorithm 8 with the same
    step (1/L from the oracle's power iteration) and iteration count."""
    reqs = []
    for n, nth, T, seed, iters in ((64, 45, 0.8, 41, 5), (96, 90, 0.9, 42, 4),
                                   (128, 45, 0.8, 43, 3), (64, 90, 1.1, 44, 6)):
        prob, c, g, it = request(n, nth, T, seed, iters=iters)
        L = o.power(c.astype(np.float64), np.ones((n, n, n)), T, nth, iters=8) if n <= 96 else 0
        reqs.append((prob, c, g, it, T, nth, 1.0 / L if L else 0.02))
    with F.Server(8 << 30, 4) as srv:
        tickets = [srv.submit(prob, c, g, 1e-3, s, it) for prob, c, g, it, _, _, s in reqs]
        done = [srv.wait(t)[0] for t in tickets]
        assert srv.stats()["completed"] == len(reqs)
    for (prob, c, g, it, T, nth, s), h in zip(reqs, done):
        if prob.n > 96:
            continue
        h_or, _, k = o.fb(c.astype(np.float64), g.astype(np.float64), T, 1e-3, s, it)
        assert k == it
        assert rel(h, h_or) < FP32_TOL, (prob.n, rel(h, h_or))


def test_invalid_requests_rejected():
    prob, c, g, iters = request(32, 12, 0.5, 41)
    with F.Server(1 << 20, 2) as srv:
        with pytest.raises(F.FFPATError):  # needs more than the 1 MiB budget
            srv.submit(prob, c, g, 1e-3, 0.02, iters)
    with F.Server(1 << 30, 2) as srv:
        with pytest.raises(F.FFPATError):
            srv.submit(F.problem(32, 0.5, 12, F.FP64), c, g, 1e-3, 0.02, iters)
        with pytest.raises(F.FFPATError):
            p33 = F.problem(33, 0.5, 12, F.FP32_KAHAN)
            srv.submit(p33, np.ones((33,) * 3), np.ones((12, 33, 33)), 1e-3, 0.02, 1)
