"""Trajectory differentiation: ``torch.autograd.Function`` over nb_run / nb_adjoint.

Forward runs `steps` paper updates with nb_run, writing a checkpoint of
(x, v) every `ckpt_every` steps into a tensor owned by the autograd context.
Backward calls nb_adjoint, which recomputes each segment from its checkpoint
and sweeps it backwards with the all-pairs vector-Jacobian product kernel,
returning gradients w.r.t. the initial positions, velocities and masses.
"""
from __future__ import annotations

import torch

from .nbody import Context


class NBodyTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, nbctx: Context, steps: int, ckpt_every: int):
        n = m.shape[0]
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        mm = m.detach().contiguous()
        ckpt = torch.empty((steps // ckpt_every + 1, n, 6), dtype=x.dtype, device=x.device)
        nbctx.run(x, v, mm, steps, ckpt=ckpt, ckpt_every=ckpt_every)
        ctx.save_for_backward(mm, ckpt)
        ctx.nbctx, ctx.steps, ctx.ckpt_every = nbctx, steps, ckpt_every
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        m, ckpt = ctx.saved_tensors
        if gx is None:
            gx = torch.zeros_like(ckpt[0, :, :3])
        if gv is None:
            gv = torch.zeros_like(ckpt[0, :, 3:])
        xb, vb, mb = ctx.nbctx.adjoint(m, ctx.steps, ckpt, ctx.ckpt_every,
                                       gx.contiguous(), gv.contiguous())
        return xb, vb, mb, None, None, None


def trajectory(x0, v0, m, nbctx: Context, steps: int, ckpt_every: int):
    """(x_T, v_T) after `steps` paper updates, differentiable in x0, v0, m."""
    return NBodyTrajectory.apply(x0, v0, m, nbctx, steps, ckpt_every)
