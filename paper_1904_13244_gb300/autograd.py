"""Differentiation form: the MR-STAT signal as a torch.autograd.Function.

forward(alpha) = s(alpha) (Algorithm 2) and backward(grad_s) = Re(J_s^H grad_s)
(Algorithm 4).  For a real-valued loss L of the complex signal, PyTorch hands the
backward the conjugate-Wirtinger gradient grad_s, and dL/dalpha = Re(J_s^H grad_s)
because alpha is real.

With ``checkpoint=k`` (a multiple of 4, default 64) the forward keeps only the
Bloch state of every voxel at every k-th TR and the backward re-runs the segments of
the recursion from those states (mrstat_forward_ckpt / mrstat_jhw_ckpt); with
``checkpoint=0`` the forward caches the full time courses and the backward streams
them (mrstat_linearize / mrstat_jhw).  Both run entirely in libmrstat.

A plan holds the state of one forward at a time: call backward before the next
forward on the same plan.
"""
from __future__ import annotations

import torch

from . import _binding as _b


class Signal(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, plan, b1=None, mask=None, checkpoint: int = 64):
        if alpha.dtype != torch.float32 or not alpha.is_cuda:
            raise TypeError("alpha must be a CUDA float32 tensor [4, nv]")
        alpha = alpha.detach().contiguous()
        s = torch.empty((plan.ntr, plan.nkx), dtype=torch.complex64, device=alpha.device)
        if checkpoint:
            _b.mrstat_forward_ckpt(plan.handle, alpha, b1, mask, int(checkpoint), s)
        else:
            _b.mrstat_linearize(plan.handle, alpha, b1, mask)
            _b.mrstat_forward(plan.handle, alpha, b1, mask, s)
        # the checkpointed backward reads alpha, b1 and mask from these buffers
        ctx.save_for_backward(alpha)
        ctx.keep = (b1, mask)
        ctx.plan = plan
        ctx.checkpoint = int(checkpoint)
        return s

    @staticmethod
    def backward(ctx, grad_s):
        plan = ctx.plan
        g = torch.empty((4, plan.nv), dtype=torch.float32, device=grad_s.device)
        w = grad_s.contiguous().to(torch.complex64)
        if ctx.checkpoint:
            _b.mrstat_jhw_ckpt(plan.handle, w, g)
        else:
            _b.mrstat_jhw(plan.handle, w, g)
        return g, None, None, None, None


def signal(alpha, plan, b1=None, mask=None, checkpoint: int = 64):
    """s(alpha) with a backward pass through libmrstat (see Signal)."""
    return Signal.apply(alpha, plan, b1, mask, checkpoint)
