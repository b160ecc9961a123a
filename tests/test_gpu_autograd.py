"""The differentiable operator: FFPATOp (torch.autograd.Function) with the
checkpointed transposed solve, against the oracle gradient and central
finite differences."""
import numpy as np
import pytest

import oracle.oracle as o
from paper_1901_06503_gb300 import build_lib
from paper_1901_06503_gb300 import ffpat as F
from paper_1901_06503_gb300.autograd import forward_op
from paper_1901_06503_gb300.inputs import config, random_data, random_speed, random_volume

from tolerances import FP32_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    F.lib()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("every", [1, 4, 16, 1000])
@pytest.mark.parametrize("n,nth,T", [(24, 6, 0.5), (32, 8, 0.03)])
def test_gradients_match_oracle_fp64(n, nth, T, every):
    c = random_speed(n, 1000 + n)
    h = random_volume(n, 1001 + n)
    w = random_data(nth, n, 1002 + n)
    prob = F.problem(n, T, nth, F.FP64)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    ct = torch.tensor(c, device="cuda", requires_grad=True)
    g = forward_op(ht, ct, prob, every)
    (g * torch.tensor(w, device="cuda")).sum().backward()
    gh_or, gc_or = o.grad(c, h, w, T)
    assert rel(g.detach().cpu().numpy(), o.forward(c, h, T, nth)) < 1e-10
    assert rel(ht.grad.cpu().numpy(), gh_or) < 1e-10
    assert rel(ct.grad.cpu().numpy(), gc_or) < 1e-10


def test_grad_h_only_uses_adjoint():
    n, nth, T = 32, 8, 0.4
    c, h, w = random_speed(n, 1), random_volume(n, 2), random_data(nth, n, 3)
    prob = F.problem(n, T, nth, F.FP64)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    g = forward_op(ht, torch.tensor(c, device="cuda"), prob)
    (g * torch.tensor(w, device="cuda")).sum().backward()
    assert rel(ht.grad.cpu().numpy(), o.adjoint(c, w, T)) < 1e-10


def test_fp32_gradient_matches_oracle_at_48():
    """The FP32 path at 48^3 (config-3 generator rescaled) against the FP64 oracle gradient."""
    wl = config(3, n=48)
    c = wl.c.astype(np.float32).astype(np.float64)
    h = wl.h.astype(np.float32).astype(np.float64)
    w = random_data(wl.n_angles, 48, 5).astype(np.float32).astype(np.float64)
    prob = F.problem(48, wl.T, wl.n_angles, F.FP32)
    ht = torch.tensor(h, device="cuda", dtype=torch.float32, requires_grad=True)
    ct = torch.tensor(c, device="cuda", dtype=torch.float32, requires_grad=True)
    g = forward_op(ht, ct, prob, 16)
    (g * torch.tensor(w, device="cuda", dtype=torch.float32)).sum().backward()
    gh_or, gc_or = o.grad(c, h, w, wl.T)
    assert rel(ht.grad.double().cpu().numpy(), gh_or) < FP32_TOL
    assert rel(ct.grad.double().cpu().numpy(), gc_or) < FP32_TOL


def test_central_differences_fp64():
    """Loss 1/2 ||A h - g||^2 on the config-3 phantom (balls, Gaussian-bump
    sound speed) at 32^3; directional derivatives in c and h against central
    differences with eps = 1e-3 (relative size of a smooth perturbation of c),
    8 random smooth directions; the maximum of c is never perturbed so that Nt
    and dt stay fixed.  The central difference must converge onto the
    analytic value at second order (its error shrinks ~4x when eps halves)."""
    from paper_1901_06503_gb300.inputs import gaussian_random_field
    wl = config(3, n=32)
    n, nth, T = 32, 12, 0.5
    rng = np.random.default_rng(9)
    c, h = wl.c, wl.h
    imax = np.unravel_index(np.argmax(c), c.shape)
    gd = torch.tensor(random_data(nth, n, 13), device="cuda")
    prob = F.problem(n, T, nth, F.FP64)

    def loss(hh, cc):
        return float(0.5 * ((forward_op(hh, cc, prob, 4) - gd) ** 2).sum())

    ht = torch.tensor(h, device="cuda", requires_grad=True)
    ct = torch.tensor(c, device="cuda", requires_grad=True)
    out = forward_op(ht, ct, prob, 4)
    (0.5 * ((out - gd) ** 2).sum()).backward()
    eps = 1e-3
    cc, hh = torch.tensor(c, device="cuda"), torch.tensor(h, device="cuda")
    with torch.no_grad():
        for i in range(8):
            d = gaussian_random_field(n, 0.3, np.random.default_rng(100 + i)) * c
            d[imax] = 0.0
            dc = torch.tensor(d, device="cuda")
            dh = torch.tensor(rng.standard_normal((n, n, n)), device="cuda")
            fd = [(loss(hh, cc + e * dc) - loss(hh, cc - e * dc)) / (2 * e) for e in (eps, eps / 2)]
            an_c = float((ct.grad * dc).sum())
            err = [abs(f - an_c) for f in fd]
            assert err[0] < 1e-2 * abs(an_c)
            assert err[1] < 0.35 * err[0] or err[0] < 1e-9 * abs(an_c)
            fd_h = (loss(hh + eps * dh, cc) - loss(hh - eps * dh, cc)) / (2 * eps)
            an_h = float((ht.grad * dh).sum())
            assert abs(fd_h - an_h) < 1e-8 * abs(an_h)


def test_config3_central_differences_fp32_192():
    """The differentiable operator as the 192^3 workload runs it: FP32,
    90 angles, T = 1, checkpoints every 16 steps, loss 1/2 ||A(c) h - g||^2
    with g = A h_true + 1 % noise and h = h_true + a smooth perturbation.
    32 random directions (dh, dc) -- smooth fields; dc vanishes wherever c is
    within reach of its maximum, so that Nt and dt (from max c) stay fixed --
    each checked against <grad_h, dh> +
    <grad_c, dc> from the hand-written FP32 backward pass:

    * central differences of the FP32 operator at eps = 1e-3 within 1 %: the
      h-part of the loss is quadratic (exact), the c-part carries the
      truncation eps^2 |d^3 L / d eps^3| / 6 (a relative speed change of 1e-3
      over the workload's shortest wavelengths and T = 1 keeps it below 1 %),
      and the FP32 rounding of the two loss values divided by 2 eps;
    * central differences of the same discretisation in FP64 at eps and
      eps / 2 converge onto the analytic value at second order (the error
      shrinks at least ~3x) until they reach the FP32 gradient's own accuracy.

    The loss differences are formed in FP64 from the residuals."""
    from paper_1901_06503_gb300.inputs import gaussian_random_field
    wl = config(3)
    n, nth, T = wl.n, wl.n_angles, wl.T
    prob = F.problem(n, T, nth, F.FP32)
    p64 = F.problem(n, T, nth, F.FP64)
    c = wl.c
    ct0 = torch.tensor(c, device="cuda", dtype=torch.float32)
    ht_true = torch.tensor(wl.h, device="cuda", dtype=torch.float32)
    with torch.no_grad():
        g = F.forward(prob, ct0, ht_true).double()
        g = g + 0.01 * float(g.norm()) / g.numel() ** 0.5 * torch.tensor(
            wl.noise, device="cuda")
    h0 = wl.h + 0.05 * gaussian_random_field(n, 0.2, np.random.default_rng(31))
    ht = torch.tensor(h0, device="cuda", dtype=torch.float32, requires_grad=True)
    ct = torch.tensor(c, device="cuda", dtype=torch.float32, requires_grad=True)
    r = forward_op(ht, ct, prob, 16).double() - g
    (0.5 * (r * r).sum()).backward()
    gh, gc = ht.grad.double(), ct.grad.double()
    # the FP32 operator sees the FP32-rounded point; the FP64 one the same point
    hh = torch.tensor(h0, device="cuda", dtype=torch.float32).double()
    cc = torch.tensor(c, device="cuda", dtype=torch.float32).double()
    ws32, ws64 = F.workspace(prob), F.workspace(p64)

    def central(e, dh, dc, fp64):
        def res(s):
            with torch.no_grad():
                if fp64:
                    return F.forward(p64, cc + s * dc, hh + s * dh, ws=ws64) - g
                return F.forward(prob, (cc + s * dc).float(), (hh + s * dh).float(),
                                 ws=ws32).double() - g
        rp, rm = res(e), res(-e)
        return float(0.5 * ((rp - rm) * (rp + rm)).sum()) / (2 * e)

    eps, errs32, errs64 = 1e-3, [], []
    for i in range(32):
        rng = np.random.default_rng(300 + i)
        dc = gaussian_random_field(n, 0.3, rng) * c
        # no perturbation where it could lift c above its maximum: Nt and dt
        # (from max c) stay those of the unperturbed problem on both sides
        dc[c > c.max() - 4 * eps * np.abs(dc).max()] = 0.0
        dh = gaussian_random_field(n, 0.15, rng)
        dct = torch.tensor(dc, device="cuda")
        dht = torch.tensor(dh, device="cuda")
        an = float((gh * dht).sum() + (gc * dct).sum())
        e32 = abs(central(eps, dht, dct, False) - an)
        assert e32 < 1e-2 * abs(an), (i, e32, an)
        e64 = abs(central(eps, dht, dct, True) - an)
        e64h = abs(central(eps / 2, dht, dct, True) - an)
        assert e64h < 0.35 * e64 or e64h < FP32_TOL * abs(an), (i, e64, e64h, an)
        errs32.append(e32 / abs(an))
        errs64.append((e64 / abs(an), e64h / abs(an)))
    print(f"config-3 FD: FP32 eps=1e-3 max rel err {max(errs32):.3e} median "
          f"{float(np.median(errs32)):.3e}; FP64 eps, eps/2 max "
          f"{max(e[0] for e in errs64):.3e}, {max(e[1] for e in errs64):.3e}")


@pytest.mark.parametrize("n,every,path", [(128, 4, 0), (128, 16, 0), (128, 5, 0), (48, 6, 3)])
def test_checkpointed_loops_two_step_bit_identical(n, every, path):
    """The checkpointed forward and the segment recomputes take two leapfrog
    steps per pass (FP32, from N = 128 or with the two-step path requested,
    checkpoints at even steps); the loss and both gradients equal those of
    the step-by-step loops bit for bit (an odd interval keeps single steps)."""
    nth, T = 8, 0.1
    c = random_speed(n, 1100 + n).astype(np.float32)
    h = random_volume(n, 1101 + n).astype(np.float32)
    w = torch.tensor(random_data(nth, n, 1102 + n), device="cuda", dtype=torch.float32)
    prob = F.problem(n, T, nth, F.FP32)
    out = {}
    try:
        for p in (path, 2):
            F.set_stencil_path(p)
            ht = torch.tensor(h, device="cuda", requires_grad=True)
            ct = torch.tensor(c, device="cuda", requires_grad=True)
            g = forward_op(ht, ct, prob, every)
            (g * w).sum().backward()
            torch.cuda.synchronize()
            out[p] = (g.detach().cpu().numpy(), ht.grad.cpu().numpy(), ct.grad.cpu().numpy())
    finally:
        F.set_stencil_path(0)
    for a, b in zip(out[path], out[2]):
        assert np.array_equal(a, b)
