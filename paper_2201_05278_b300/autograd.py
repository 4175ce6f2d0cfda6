"""torch.autograd entry to the misfit gradient: marshalling around sw_gradient.

    J = misfit(velocity, grid, observed, n_steps)            # scalar tensor
    J.backward()                                               # velocity.grad = dJ/dc
    J = misfit(velocity, grid, observed, n_steps, density=rho)
    J.backward()                                               # and rho.grad = dJ/drho

The forward call sets the model on the grid (sw_set_model) and runs
sw_gradient, which returns the misfit, dJ/dc and (with a density) dJ/drho of
the exact discrete adjoint; backward scales them by the incoming gradient of
J.  Everything runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import api


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, velocity, density, grid, observed, n_steps, checkpoint_every, checkpoint_format):
        vel = velocity.detach().contiguous()
        rho = None if density is None else density.detach().to(device=vel.device, dtype=torch.float32).contiguous()
        api.sw_set_model(grid, vel, rho)
        grad = torch.empty_like(vel)
        grad_rho = None if rho is None else torch.empty_like(rho)
        obs = observed.detach().to(device=vel.device, dtype=torch.float32).contiguous()
        j = api.sw_gradient(grid, int(n_steps), obs, grad, int(checkpoint_every), int(checkpoint_format),
                            grad_rho=grad_rho)
        ctx.has_rho = grad_rho is not None
        ctx.save_for_backward(grad, grad_rho if grad_rho is not None else grad)
        return torch.tensor(j, dtype=torch.float64, device=vel.device)

    @staticmethod
    def backward(ctx, grad_j):
        grad, grad_rho = ctx.saved_tensors
        s = grad_j.to(grad.dtype)
        return grad * s, (grad_rho * s if ctx.has_rho else None), None, None, None, None, None


def misfit(velocity: torch.Tensor, grid: api.Grid, observed: torch.Tensor, n_steps: int,
           checkpoint_every: int = 0, checkpoint_format: int = api.SW_CKPT_FP32,
           density: torch.Tensor = None) -> torch.Tensor:
    """J = 1/2 |d(velocity[, density]) - observed|^2 of a forward run on `grid`
    (whose acquisition is set), differentiable with respect to `velocity` and
    `density`."""
    return _Misfit.apply(velocity, density, grid, observed, n_steps, checkpoint_every, checkpoint_format)
