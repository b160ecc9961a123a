"""torch.autograd.Function over the forward operator g = P W(c) h.

Forward calls ffpat_forward (or, when c needs a gradient, ffpat_forward_ckpt,
which keeps wavefield checkpoints every `every` steps); backward is the
hand-written transposed solve: ffpat_adjoint for grad_h alone, or
ffpat_backward, which recomputes each checkpoint segment and also returns the
sound-speed gradient (dt held fixed).  Argument marshalling only; every step
runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import ffpat as F


class FFPATOp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, c, prob, every=16):
        ctx.prob = prob
        ctx.every = int(every)
        ctx.ws = F.workspace(prob, h.device)
        need_c = bool(ctx.needs_input_grad[1])
        if need_c:
            nt, _, _ = F.problem_info(prob, float(c.max().item()))
            ctx.ckpt = torch.empty(F.ckpt_bytes(prob, nt, every), dtype=torch.uint8,
                                   device=h.device)
            g = F.forward_ckpt(prob, c, h, every, ctx.ckpt, ws=ctx.ws)
        else:
            ctx.ckpt = None
            g = F.forward(prob, c, h, ws=ctx.ws)
        ctx.save_for_backward(c)
        return g

    @staticmethod
    def backward(ctx, grad_g):
        (c,) = ctx.saved_tensors
        grad_g = grad_g.contiguous()
        want_h, want_c = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gh = gc = None
        if want_c:
            gh, gc = F.backward(ctx.prob, c, grad_g, ctx.every, ctx.ckpt, want_h=want_h,
                                want_c=True, ws=ctx.ws)
        elif want_h:
            gh = F.adjoint(ctx.prob, c, grad_g, ws=ctx.ws)
        return gh, gc, None, None


def forward_op(h: torch.Tensor, c: torch.Tensor, prob: F.Problem, every: int = 16) -> torch.Tensor:
    """Differentiable g = P W(c) h (gradients for h and c)."""
    return FFPATOp.apply(h, c, prob, every)
