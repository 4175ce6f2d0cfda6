"""Misfit gradient over many shots, partitioned across processes.

The paper names full-waveform inversion as the solver's use (Sec. 1 and 6).
Its objective is a sum over shots, J = sum_s J_s, and so is its gradient;
every shot is an independent forward and adjoint simulation.  Under
torch.distributed (one process per GPU) rank r of N takes the shots
r, r + N, r + 2N, ..., computes their summed misfit and gradient on its own
device with one sw_gradient_shots call, and a single all-reduce (sum) of the
misfit and the gradient tensors gives every rank the totals.  The
simulations never exchange anything else.  Without a process group the
same call runs every shot in this process.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np


def shots_of_rank(n_shots: int, world: int, rank: int) -> List[int]:
    """The shots rank `rank` of `world` runs: rank, rank + world, ... (each shot on exactly one rank)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return list(range(rank, n_shots, world))


def _group_info(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def reduce_sum(misfit: float, tensors: Sequence, group=None) -> float:
    """Sums the misfit and, in place, every tensor over the ranks of `group`
    (all-reduce; NCCL for CUDA tensors, gloo for CPU tensors).  Returns the
    summed misfit.  Without a process group nothing changes."""
    world, _ = _group_info(group)
    if world == 1:
        return float(misfit)
    import torch
    import torch.distributed as dist
    dev = tensors[0].device if tensors else torch.device("cpu")
    j = torch.tensor([float(misfit)], dtype=torch.float64, device=dev)
    dist.all_reduce(j, op=dist.ReduceOp.SUM, group=group)
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(j.item())


def partitioned_gradient(n_shots: int, local: Callable[[List[int]], Tuple[float, list]], group=None):
    """local(shots) returns (misfit, [gradient tensors]) summed over the given
    shot indices (zeros for an empty list); this rank runs its share of the
    shots and the sums are reduced over the group.  Returns (J, tensors)."""
    world, rank = _group_info(group)
    mine = shots_of_rank(n_shots, world, rank)
    j, tensors = local(mine)
    return reduce_sum(j, tensors, group), tensors


def misfit_gradient(g, shot_src_pos, observed, n_steps: int, checkpoint_every: int = 0, checkpoint_format: int = 0,
                    density: bool = False, group=None):
    """J and dJ/dc (and dJ/drho with density=True) summed over every shot, on
    the grid `g` of this rank's device (its model and acquisition set; the
    acquisition's sources are moved to each shot's positions).

      shot_src_pos  [n_shots][n_src][ndim] (or [n_shots][ndim]) positions, metres
      observed      [n_shots][n_steps][n_rec] data, a tensor on g's device or
                    on the host (only this rank's shots are read)

    Returns (J, grad_vel) or (J, grad_vel, grad_rho) as tensors on g's device;
    every rank gets the same totals."""
    import torch
    from . import api
    pos = np.asarray(shot_src_pos, dtype=np.float64)
    n_shots = int(pos.shape[0])
    dev = torch.device("cuda", torch.cuda.current_device())

    def local(mine):
        gv = torch.zeros(g.shape, dtype=torch.float32, device=dev)
        gr = torch.zeros(g.shape, dtype=torch.float32, device=dev) if density else None
        if not mine:
            return 0.0, [gv] + ([gr] if density else [])
        obs = observed[mine] if hasattr(observed, "index_select") else np.ascontiguousarray(np.asarray(observed)[mine])
        if hasattr(obs, "contiguous"):
            obs = obs.contiguous()
        j = api.sw_gradient_shots(g, pos[mine], n_steps, obs, gv, checkpoint_every, checkpoint_format, grad_rho=gr)
        return j, [gv] + ([gr] if density else [])

    j, tensors = partitioned_gradient(n_shots, local, group)
    return (j,) + tuple(tensors)
