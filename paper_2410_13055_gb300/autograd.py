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
        torch.cuda.current_stream().synchronize()
        h = net.array("h")
        w = torch.tensor([sc_w for sc_w in net.weights], dtype=torch.float64, device=h.device)
        if batch is not None:
            mask = torch.zeros_like(w)
            mask[list(batch)] = 1.0
            w = w * mask * (net.weights.sum() / float(sum(net.weights[list(batch)])))
        val = (h * w).sum()
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
