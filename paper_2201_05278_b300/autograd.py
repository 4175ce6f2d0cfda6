"""torch.autograd entry to the misfit gradient: marshalling around sw_gradient.

    J = misfit(velocity, grid, observed, n_steps)   # scalar tensor
    J.backward()                                      # velocity.grad = dJ/dc

The forward call sets the velocity model on the grid (sw_set_model) and runs
sw_gradient, which returns the misfit and dJ/dc of the exact discrete
adjoint (constant density); backward scales that gradient by the incoming
gradient of J.  Everything runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import api


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, velocity, grid, observed, n_steps, checkpoint_every, checkpoint_format):
        vel = velocity.detach().contiguous()
        api.sw_set_model(grid, vel)
        grad = torch.empty_like(vel)
        obs = observed.detach().to(device=vel.device, dtype=torch.float32).contiguous()
        j = api.sw_gradient(grid, int(n_steps), obs, grad, int(checkpoint_every), int(checkpoint_format))
        ctx.save_for_backward(grad)
        return torch.tensor(j, dtype=torch.float64, device=vel.device)

    @staticmethod
    def backward(ctx, grad_j):
        (grad,) = ctx.saved_tensors
        return (grad * grad_j.to(grad.dtype)), None, None, None, None, None


def misfit(velocity: torch.Tensor, grid: api.Grid, observed: torch.Tensor, n_steps: int,
           checkpoint_every: int = 0, checkpoint_format: int = api.SW_CKPT_FP32) -> torch.Tensor:
    """J = 1/2 |d(velocity) - observed|^2 of a forward run on `grid` (whose
    acquisition is set), differentiable with respect to `velocity`."""
    return _Misfit.apply(velocity, grid, observed, n_steps, checkpoint_every, checkpoint_format)
