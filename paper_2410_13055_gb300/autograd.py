"""torch.autograd wrapper of the planner's operating objective (Eq. 1, Section 2.2).

``planner_objective(eta, net)`` returns sum_s w_s h_s(x*_s(eta)) for the scenarios of
``net`` (a ``gx.Network``); its backward is the implicit gradient computed by the
adjoint message passing of ``gx_dispatch_grad_batch``.  The dispatch solution stays in
the network's workspace between forward and backward: no solver iterate is kept, only
the solved state (the adjoint re-derives the active set from it).
"""
from __future__ import annotations

import torch

from . import gx


class PlannerObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eta, net, batch, warm):
        net.solve(eta, batch=batch, warm=warm)
        # sum_s w'_s h_s, computed by the library (GX_ARR_OBJ); copied out of the workspace
        val = net.array("obj")[0].clone()
        ctx.net = net
        ctx.warm = warm
        ctx.save_for_backward(eta)
        return val.to(eta.dtype)

    @staticmethod
    def backward(ctx, gout):
        (eta,) = ctx.saved_tensors
        g = ctx.net.grad(eta.detach().contiguous(), warm=ctx.warm)
        return gout * g, None, None, None


def planner_objective(eta, net: "gx.Network", batch=None, warm="cold"):
    """sum_s w'_s h_s at plan eta (FP32 CUDA tensor [K]); differentiable in eta."""
    return PlannerObjective.apply(eta, net, batch, warm)
