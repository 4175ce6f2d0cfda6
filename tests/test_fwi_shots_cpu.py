"""The shot partition of the multi-shot misfit gradient on CPU.

Two gloo ranks split four shots (rank r takes shots r, r + 2) and sum their
misfits and gradients with one all-reduce; the FP64 adjoint oracle stands in
for the per-shot GPU gradient (the partition and the reduction are the
host-side logic under test).  Both ranks must end with the single-process sum
over all shots, and every shot must run on exactly one rank.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2201_05278_b300 import fwi

N_SHOTS = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import oracle
    rng = np.random.default_rng(8)
    shape, spacing, order, n = (30, 34), (10.0, 10.0), 4, 70
    v_true = 1800.0 + 600.0 * rng.random(shape)
    v0 = np.full(shape, 2000.0)
    dt = 0.35 * 10.0 / v_true.max()
    wav = np.asarray(oracle.ricker_samples(25.0, dt, n), dtype=np.float64)
    shots = [(40.0 + 35.0 * k, 60.0 + 20.0 * k) for k in range(N_SHOTS)]
    rec = [(30.0, 50.0), (30.0, 150.0), (120.0, 220.0)]
    kw = dict(rec_pos=rec, nbl=[0, 5, 5, 5], bc=["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet"],
              damp_alpha=2.0, damp_degree=3, window_radius=3)
    obs = [oracle.forward(2, shape, spacing, order, v_true, dt, n, src_pos=[s], wavelet=wav, **kw)[0] for s in shots]
    return shape, spacing, order, v0, dt, n, wav, shots, obs, kw


def _local_oracle(case, log=None):
    from oracle import adjoint as A
    import torch
    shape, spacing, order, v0, dt, n, wav, shots, obs, kw = case

    def local(mine):
        if log is not None:
            log.extend(mine)
        J, g = 0.0, np.zeros(shape)
        for s in mine:
            pb = A.make_problem(2, shape, spacing, order, v0, dt, src_pos=[shots[s]], **kw)
            j, gc, _ = A.adjoint_gradient(pb, wav, obs[s], n)
            J += j
            g += gc
        return J, [torch.from_numpy(g)]
    return local


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ran = []
        J, (g,) = fwi.partitioned_gradient(N_SHOTS, _local_oracle(_case(), ran))
        out[rank] = (J, g.numpy(), ran)
    finally:
        dist.destroy_process_group()


def test_shots_of_rank_cover_every_shot_once():
    for n_shots in (1, 4, 7, 16):
        for world in (1, 2, 3, 5):
            got = sorted(s for r in range(world) for s in fwi.shots_of_rank(n_shots, world, r))
            assert got == list(range(n_shots))
    with pytest.raises(ValueError):
        fwi.shots_of_rank(4, 2, 2)


def test_two_ranks_sum_to_the_single_process_gradient():
    case = _case()
    J_all, (g_all,) = fwi.partitioned_gradient(N_SHOTS, _local_oracle(case))  # no process group: every shot
    J_parts = [_local_oracle(case)([s])[0] for s in range(N_SHOTS)]
    assert J_all == pytest.approx(sum(J_parts), rel=1e-12)
    assert all(j > 0 for j in J_parts)
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res[0][2] + res[1][2]) == list(range(N_SHOTS))
    assert res[0][2] == [0, 2] and res[1][2] == [1, 3]
    g_ref = g_all.numpy()
    for r in range(world):
        J, g, _ = res[r]
        assert J == pytest.approx(J_all, rel=1e-12)
        assert np.allclose(g, g_ref, rtol=0, atol=1e-12 * np.abs(g_ref).max())
    assert np.abs(g_ref).max() > 0
