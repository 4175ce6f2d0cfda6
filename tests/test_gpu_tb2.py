"""Temporal blocking (SW_STENCIL_TB2): two leapfrog steps per launch on 2D grids.

Every node value is formed by the per-step kernels' operations in the same
order, so the wavefield levels must equal the plain per-step 2D kernels' bit
for bit (the two sources of these cases share no node); the seismograms come
from another receiver sampler and agree to rounding.  Both match the FP64
oracle within the FP32 bars.  Covered: every space order, odd and even step
counts (an odd last step runs on the per-step kernels), ragged tiles, mixed
face conditions with sources and receivers next to the faces and in the
absorbing layers, host buffers, the launch count and graph replay.
"""
import dataclasses

import numpy as np
import pytest

from paper_2201_05278_b300 import api
from tests.harness import assert_parity, rel_l2, run_gpu, run_oracle
from tests.test_gpu_parity import small_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
def test_two_step_kernel_equals_the_per_step_kernels(cuda_device, order):
    w = small_case(2, order, False, seed=200 + order, n_steps=61)
    s_tb, p_tb = run_gpu(w, variant=api.SW_STENCIL_TB2, expect_variant=api.SW_STENCIL_TB2)
    s_pl, p_pl = run_gpu(w, variant=api.SW_STENCIL_PLAIN, expect_variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(p_tb, p_pl)
    assert rel_l2(s_tb, s_pl) <= 1e-6
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_tb, s_ref, "seismogram")
    assert_parity(p_tb, p_ref, "field")


@pytest.mark.parametrize("n_steps", [0, 1, 2, 3, 4, 37, 64])
def test_two_step_kernel_step_counts(cuda_device, n_steps):
    w = small_case(2, 8, False, seed=5, n_steps=max(n_steps, 1))
    s_tb, p_tb = run_gpu(w, n_steps=n_steps, variant=api.SW_STENCIL_TB2)
    s_pl, p_pl = run_gpu(w, n_steps=n_steps, variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(p_tb, p_pl)
    assert s_tb.shape == s_pl.shape
    if n_steps:
        assert rel_l2(s_tb, s_pl) <= 1e-6 or np.abs(s_pl).max() == 0


@pytest.mark.parametrize("faces", [0, 1, 2])
def test_two_step_kernel_faces_and_ragged_tiles(cuda_device, faces):
    """Grids not a multiple of the 32 x 64 tile, sources and receivers next to
    Dirichlet and Neumann faces and deep in the absorbing layers."""
    w = small_case(2, 8, False, seed=17 + faces, n_steps=90)
    shape = [(70, 131), (33, 65), (97, 203)][faces]
    rng = np.random.default_rng(faces)
    vel = (1800.0 + 900.0 * rng.random(shape)).astype(np.float32)
    bcs = [["null_dirichlet", "null_neumann", "null_neumann", "null_dirichlet"],
           ["null_neumann", "null_dirichlet", "null_dirichlet", "none"],
           ["null_dirichlet", "null_dirichlet", "null_neumann", "null_neumann"]][faces]
    nbl = [[0, 6, 5, 0], [4, 3, 0, 7], [6, 0, 0, 5]][faces]
    h = w.spacing
    phys = [(shape[a] - nbl[2 * a] - nbl[2 * a + 1] - 1) * h[a] for a in range(2)]
    src = np.array([[0.6 * h[0] - nbl[0] * h[0] + 3.2 * h[0], 0.45 * phys[1]],
                    [0.5 * phys[0], (shape[1] - nbl[2] - 4.3) * h[1]]])
    rec = np.array([[(3.5 - nbl[0]) * h[0], 0.3 * phys[1]], [0.7 * phys[0], (-nbl[2] + 3.6) * h[1]],
                    [(shape[0] - nbl[0] - 4.1) * h[0], 0.8 * phys[1]]])
    w = dataclasses.replace(w, shape=shape, velocity=vel, bc=bcs, nbl=nbl, src_pos=src, rec_pos=rec,
                            dt=0.3 * min(h) / float(vel.max()))
    s_tb, p_tb = run_gpu(w, variant=api.SW_STENCIL_TB2, expect_variant=api.SW_STENCIL_TB2)
    s_pl, p_pl = run_gpu(w, variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(p_tb, p_pl)
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_tb, s_ref, "seismogram")
    assert_parity(p_tb, p_ref, "field")


def test_two_step_kernel_launches_replay_and_host_buffers(cuda_device):
    """Per two steps: the two-step launch, a face pass per level (with the
    receivers) and step n+1's sources; the second call replays a captured graph
    with the same result; host output buffers give the same values."""
    w = small_case(2, 8, False, seed=9, n_steps=40)
    s1, p1, prof = run_gpu(w, variant=api.SW_STENCIL_TB2, profile=True)
    assert prof[1] == 20  # two-step launches timed (profiling every launch)
    assert prof[2] == 20 * 4 + 1  # + the final-field copy
    s2, p2 = run_gpu(w, variant=api.SW_STENCIL_TB2, device_io=False)
    assert np.array_equal(p1, p2) and np.array_equal(s1, s2)
    import torch
    g = api.sw_create_grid(2, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).cuda())
        api.sw_set_stencil_variant(g, api.SW_STENCIL_TB2)
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        runs = []
        for _ in range(3):  # direct, captured, replayed
            seis = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device="cuda:0")
            fin = torch.zeros(w.shape, dtype=torch.float32, device="cuda:0")
            api.sw_forward(g, w.n_steps, seis, fin)
            runs.append((seis.cpu().numpy(), fin.cpu().numpy()))
        for s, p in runs[1:]:
            assert np.array_equal(s, runs[0][0]) and np.array_equal(p, runs[0][1])
        assert np.array_equal(runs[0][1], p1)
    finally:
        g.close()


def test_two_step_kernel_is_2d_only(cuda_device):
    w3 = small_case(3, 8, False, n_steps=10)
    g = api.sw_create_grid(3, w3.shape, w3.spacing, 8, w3.nbl, w3.bc, 0.0, 3, 0.0)
    try:
        with pytest.raises(api.SimwaveError) as e:
            api.sw_set_stencil_variant(g, api.SW_STENCIL_TB2)
        assert e.value.status == api.SW_EINVAL
    finally:
        g.close()


def test_auto_picks_the_two_step_kernel_on_large_2d_grids(cuda_device):
    """From 4M nodes on (fields beyond L2) the default variant is the two-step
    kernel; smaller 2D grids keep the cluster run or the per-step kernels, and
    an explicit SW_STENCIL_PLAIN is honoured."""
    import torch
    for shape, big in (((2048, 2048), True), ((1024, 1024), False)):
        g = api.sw_create_grid(2, shape, (5.0, 5.0), 8, [0, 10, 10, 10],
                               ["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet"], 1.0, 3, 0.0)
        try:
            api.sw_set_model(g, torch.full(shape, 2000.0, dtype=torch.float32, device="cuda:0"))
            v = api.sw_get_stencil_variant(g)
            assert (v == api.SW_STENCIL_TB2) == big
            api.sw_set_stencil_variant(g, api.SW_STENCIL_PLAIN)
            assert api.sw_get_stencil_variant(g) == api.SW_STENCIL_PLAIN
        finally:
            g.close()
