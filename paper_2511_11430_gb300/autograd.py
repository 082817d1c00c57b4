"""Differentiable particle -> point velocity (Eq. 2-4) through the hand-written adjoint.

``VPMInduce.apply(pos, strength, tgt, sigma, compensated)`` returns u [3, n_tgt];
its backward calls ``vpm_induce_backward``, which recomputes every pair term from
the saved inputs (pos, strength, tgt only) and returns dL/dx and dL/dGamma of the
particles.  Gradients flow to pos[:, :3] and strength[:, :3]; the volume lane and
the evaluation points receive none.
"""
from __future__ import annotations

import torch

from . import api


class VPMInduce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, strength, tgt, sigma, compensated=True):
        u = api.induce(pos, strength, tgt, sigma, compensated=compensated, grad=False)
        ctx.save_for_backward(pos, strength, tgt)
        ctx.sigma = float(sigma)
        ctx.compensated = bool(compensated)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        pos, strength, tgt = ctx.saved_tensors
        dx, dG = api.induce_backward(pos, strength, tgt, ctx.sigma, grad_u.contiguous(), ctx.compensated)
        gpos = gstr = None
        if ctx.needs_input_grad[0]:
            gpos = torch.zeros_like(pos)
            gpos[:, :3] = dx.t()
        if ctx.needs_input_grad[1]:
            gstr = torch.zeros_like(strength)
            gstr[:, :3] = dG.t()
        return gpos, gstr, None, None, None


def induce(pos, strength, tgt, sigma, compensated=True):
    """Autograd-aware velocity at tgt (planar [3, n_tgt])."""
    return VPMInduce.apply(pos, strength, tgt, sigma, compensated)
