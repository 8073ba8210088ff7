"""torch.autograd wrapper of the tree force (argument marshalling only).

``long_range_force(pos, mass, context)`` builds the tree for ``pos`` (3, n)
float64 and ``mass`` (n,) float64 and returns the soft acceleration (3, n)
float32 (p3t_build_tree + p3t_long_force).  Its backward pass calls
p3t_long_force_vjp: the gradient of the tree force with the tree structure
and interaction sets of the forward pass held fixed, recomputing the
interaction sets by walking the same tree.
"""
from __future__ import annotations

import torch

from .binding import Context


class LongRangeForce(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, mass, context: Context):
        context.build_tree(pos.detach().contiguous(), mass.detach().contiguous())
        acc = context.long_force()
        fctx.context = context
        fctx.build_id = context.build_id
        return acc

    @staticmethod
    def backward(fctx, grad_acc):
        context = fctx.context
        if context.build_id != fctx.build_id:
            raise RuntimeError("the context was rebuilt between the forward "
                               "and the backward pass")
        w = grad_acc.detach().to(torch.float32).contiguous()
        gpos, gmass = context.long_force_vjp(w)
        return gpos, gmass, None


def long_range_force(pos, mass, context: Context):
    """Differentiable soft acceleration (3, n) float32 of the tree."""
    return LongRangeForce.apply(pos, mass, context)
