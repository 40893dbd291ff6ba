"""torch.autograd wrapper: J[u] as a differentiable function of the controls.

Forward evaluates J through ``ism_evaluate`` (Algorithm 1 steps (a)-(b) only); backward calls
``ism_gradient``, which recomputes the global trajectories and returns dJ/du by Theorem 2 (the
sub-problem gradients at phi = phi^u, scaled by beta_n), all in the library's kernels.  Nothing is
kept between the two calls but u: the forward states are recomputed per segment by the backward
pass instead of being stored.
"""
from __future__ import annotations

import torch

from .abi import Plan

__all__ = ["ISMObjective", "objective"]


class ISMObjective(torch.autograd.Function):
    """J = ISMObjective.apply(u, plan); u: (batch, Nt) float64 CUDA tensor, J: (batch,)."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, plan: Plan) -> torch.Tensor:
        if u.dtype != torch.float64 or not u.is_cuda:
            raise TypeError("u must be a float64 CUDA tensor of shape (batch, Nt)")
        u = u.detach().contiguous()
        J = torch.empty(plan.batch, dtype=torch.float64, device=u.device)
        with torch.cuda.device(u.device):
            torch.cuda.current_stream().synchronize()   # u is complete before the plan's stream reads it
            plan.ism_evaluate(u, J, None)
        ctx.plan = plan
        ctx.save_for_backward(u)
        return J

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (u,) = ctx.saved_tensors
        grad = torch.empty_like(u)
        with torch.cuda.device(u.device):
            torch.cuda.current_stream().synchronize()
            ctx.plan.ism_gradient(u, grad, None)
        return gJ.reshape(-1, 1).to(grad.dtype) * grad, None


def objective(u: torch.Tensor, plan: Plan) -> torch.Tensor:
    return ISMObjective.apply(u, plan)
