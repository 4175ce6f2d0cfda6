"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: relative L2 error of the seismogram and of the final field at most
1e-5 (FP32 forward vs FP64 oracle).  Small odd-shaped grids cover every
space order, both dimensions, both density paths, ragged tiles and mixed
face conditions; the named workloads are checked at full grid size with a
reduced step count, and full-length runs are checked by properties that
hold at any size (causality against the oracle's prefix, exact time-shift
invariance, amplitude scaling up to FP32 rounding noise).
"""
import numpy as np
import pytest

from paper_2201_05278_b300 import api, workloads
from paper_2201_05278_b300.workloads import Workload
from tests.harness import FP32_SEIS_TOL, assert_parity, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# Face slabs are compared against their own norm and peak, about a hundred
# times smaller than the field's: the bar there is relative to the local
# amplitude (a wrong face row or ghost image is an error of order one there;
# FP32 rounding measured 8e-6 at most on the full-grid runs).
FACE_TOL = 5e-5


def small_case(ndim, order, density, seed=0, n_steps=60):
    rng = np.random.default_rng(seed)
    r = order // 2
    if ndim == 2:
        shape = (41 + r, 57 + 3 * r)
        spacing = (7.0, 9.0)
        nbl = [0, 6, 5, 7]
        bc = ["null_neumann", "null_dirichlet", "none", "null_dirichlet"]
    else:
        shape = (23 + r, 19 + 2 * r, 37 + r)
        spacing = (9.0, 8.0, 10.0)
        nbl = [0, 4, 3, 5, 4, 6]
        bc = ["null_neumann", "null_dirichlet", "null_dirichlet", "none", "null_neumann", "null_dirichlet"]
    vel = (1800.0 + 900.0 * rng.random(shape)).astype(np.float32)
    rho = (1500.0 + 1200.0 * rng.random(shape)).astype(np.float32) if density else None
    dt = 0.3 * min(spacing) / float(vel.max())
    phys = [(shape[a] - nbl[2 * a] - nbl[2 * a + 1] - 1) * spacing[a] for a in range(ndim)]
    rw = min(4, r + 1)
    # one off-grid source, one on-grid source; receivers on and off grid
    src = np.array([[0.31 * p for p in phys], [round(0.6 * p / s) * s for p, s in zip(phys, spacing)]])
    rec = np.array([[0.5 * p for p in phys], [0.2 * p + 0.37 for p in phys], [0.8 * p for p in phys],
                    [spacing[0]] + [0.45 * p for p in phys[1:]]])
    return Workload("small", ndim, shape, spacing, order, nbl, bc, 40.0 / (max(nbl) ** 3), 3, dt, n_steps,
                    30.0, 1.0 / 30.0, src, rec, rw, vel, rho)


@pytest.mark.parametrize("density", [False, True])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
def test_small_grids_all_orders(cuda_device, ndim, order, density):
    w = small_case(ndim, order, density, seed=order + 7 * ndim)
    s_gpu, p_gpu = run_gpu(w)
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")


@pytest.mark.parametrize("density", [False, True])
@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
def test_3d_both_stencil_kernels(cuda_device, order, density):
    """The TMA-pipelined kernel (chosen automatically in 3D, constant or variable
    density) and the shared-memory-plane kernel both match the oracle."""
    w = small_case(3, order, density, seed=100 + order)
    s_ref, p_ref = run_oracle(w)
    s_tma, p_tma = run_gpu(w, expect_variant=api.SW_STENCIL_TMA)
    s_pl, p_pl = run_gpu(w, variant=api.SW_STENCIL_PLAIN, expect_variant=api.SW_STENCIL_PLAIN)
    for s, p in ((s_tma, p_tma), (s_pl, p_pl)):
        assert_parity(s, s_ref, "seismogram")
        assert_parity(p, p_ref, "field")


@pytest.mark.parametrize("order,bcs", [(2, 0), (8, 0), (8, 1), (14, 1), (20, 0)])
def test_2d_cluster_run_matches_the_plain_kernels(cuda_device, order, bcs):
    """The cluster-resident 2D run (the whole forward in one launch of one
    thread-block cluster, chosen automatically for 2D grids that fit) gives the
    plain per-step 2D kernels' seismogram and final field bit for bit, with
    sources on faces and in the absorbing layers, and matches the oracle."""
    import dataclasses
    w = small_case(2, order, False, seed=40 + order, n_steps=70)
    if bcs == 1:  # every face kind, sources next to a Dirichlet and a Neumann face
        h = w.spacing
        src = np.array([[0.7 * h[0], 0.4 * (w.shape[1] - 11) * h[1]],
                        [0.5 * (w.shape[0] - 7) * h[0], -0.5 * h[1]]])
        w = dataclasses.replace(w, bc=["null_dirichlet", "null_neumann", "null_neumann", "null_dirichlet"],
                                nbl=[3, 0, 4, 6], src_pos=src)
    s_pl, p_pl = run_gpu(w, variant=api.SW_STENCIL_PLAIN, expect_variant=api.SW_STENCIL_PLAIN)
    s_cl, p_cl, prof = run_gpu(w, profile=True, expect_variant=api.SW_STENCIL_CLUSTER)
    assert np.array_equal(s_cl, s_pl) and np.array_equal(p_cl, p_pl)
    assert prof[2] == 2  # the run and the final-field copy
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_cl, s_ref, "seismogram")
    assert_parity(p_cl, p_ref, "field")


def test_2d_cluster_run_edge_cases(cuda_device):
    """Zero and one step, host buffers, and a grid whose bands hold one row each."""
    import dataclasses
    w = small_case(2, 8, False, seed=3, n_steps=30)
    for n in (0, 1):
        s, p = run_gpu(w, n_steps=n, variant=api.SW_STENCIL_CLUSTER)
        s2, p2 = run_gpu(w, n_steps=n, variant=api.SW_STENCIL_PLAIN)
        assert np.array_equal(s, s2) and np.array_equal(p, p2)
    s, p = run_gpu(w, device_io=False, expect_variant=api.SW_STENCIL_CLUSTER)
    s2, p2 = run_gpu(w, variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(s, s2) and np.array_equal(p, p2)
    # 14 rows on up to 16 CTAs: one row per band, every halo row from other CTAs
    vel = w.velocity[:14, :]
    h = w.spacing
    small = dataclasses.replace(w, shape=(14, w.shape[1]), velocity=vel, nbl=[0, 2, 5, 7],
                                src_pos=np.array([[5.3 * h[0], 11.6 * h[1]]]),
                                rec_pos=np.array([[2.0 * h[0], 3.3 * h[1]], [6.5 * h[0], 20.0 * h[1]]]),
                                window_radius=3)
    s, p = run_gpu(small, expect_variant=api.SW_STENCIL_CLUSTER)
    s2, p2 = run_gpu(small, variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(s, s2) and np.array_equal(p, p2)
    s_ref, p_ref = run_oracle(small)
    assert_parity(s, s_ref, "seismogram")
    assert_parity(p, p_ref, "field")
    # windows of radius 5: off-grid receivers have ten rows with a non-zero
    # weight, more than the run keeps in registers (the general sampling loop)
    wide = dataclasses.replace(w, window_radius=5)
    s, p = run_gpu(wide, expect_variant=api.SW_STENCIL_CLUSTER)
    s2, p2 = run_gpu(wide, variant=api.SW_STENCIL_PLAIN)
    assert np.array_equal(s, s2) and np.array_equal(p, p2)


def test_tma_kernel_many_segments(cuda_device):
    """A grid with more work items than CTAs of one tile: segments start and end at
    every plane offset and cross tile boundaries (ragged in x, y and z)."""
    w = workloads.make("3d_layered_256", shape=(29, 70, 97), n_steps=120)
    s_ref, p_ref = run_oracle(w)
    s, p = run_gpu(w, expect_variant=api.SW_STENCIL_TMA)
    assert np.abs(s_ref).max() > 0
    assert_parity(s, s_ref, "seismogram")
    assert_parity(p, p_ref, "field")


@pytest.mark.parametrize("damp_scale", [1.0, 100.0])
def test_sources_in_the_absorbing_layers(cuda_device, damp_scale):
    """Sources whose windows reach into the absorbing layers, on the pipelined path.
    With eta dt below 1/2 at every source window node (damp_scale 1) each step's
    source increments enter through the level the step reads as p[n-1], divided
    by 1 - eta dt, inside the previous step's face launch (two launches per
    step); with damping strong enough to pass 1/2 there (damp_scale 100),
    through a launch of their own after the stencil (three per step).  Both
    match the oracle (Eq. 7, Eq. 11)."""
    import dataclasses
    w = small_case(3, 8, False, seed=5, n_steps=70)
    h = w.spacing
    # off-grid sources: one in the x- layer (node 3.5 of a 4-cell layer), one in
    # the z+ layer (node nz - 4.5 of 4 cells), one in the physical box; the
    # deepest window node of each lies 4 cells into a layer (window radius 4)
    src = np.array([[0.5 * (w.shape[0] - 5) * h[0], 0.5 * (w.shape[1] - 9) * h[1], -0.5 * h[2]],
                    [(w.shape[0] - 4.5) * h[0], 0.43 * (w.shape[1] - 9) * h[1], 0.37 * (w.shape[2] - 11) * h[2]],
                    [0.3 * (w.shape[0] - 5) * h[0], 0.6 * (w.shape[1] - 9) * h[1], 0.55 * (w.shape[2] - 11) * h[2]]])
    w = dataclasses.replace(w, src_pos=src, damp_alpha=w.damp_alpha * damp_scale)
    assert w.window_radius == 4
    e_src = w.damp_alpha * 4.0 ** w.damp_degree * w.dt  # eta dt = alpha d^p dt, d in cells
    assert (e_src < 0.5) == (damp_scale == 1.0)
    s_gpu, p_gpu, prof = run_gpu(w, profile=True, expect_variant=api.SW_STENCIL_TMA)
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")
    # per forward: the tap table, the final-field copy and (first path) step 0's
    # sources into p[-1]; per step: the stencil, the face launch (and the injection)
    if damp_scale == 1.0:
        assert prof[2] == 2 * w.n_steps + 3
    else:
        assert prof[2] == 3 * w.n_steps + 2


def test_host_and_device_buffers_agree(cuda_device):
    w = small_case(3, 8, True, seed=3, n_steps=30)
    s_dev, p_dev = run_gpu(w, device_io=True)
    s_host, p_host = run_gpu(w, device_io=False)
    assert np.array_equal(s_dev, s_host) and np.array_equal(p_dev, p_host)


def test_2d_homogeneous_full_length(cuda_device):
    w = workloads.make("2d_homogeneous_256")
    s_gpu, p_gpu = run_gpu(w)
    s_ref, p_ref = run_oracle(w)
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")


def face_sources(w):
    """Two sources in the absorbing layers near opposite corners (3.4 to 4.6 cells
    from the z+, y-, x- faces and from the z-, y+, x+ faces) plus the workload's
    own, and a 25 Hz wavelet with its energy in the first 40 ms, so that a short
    run drives every face and every layer of the full grid."""
    import dataclasses
    nz, ny, nx = w.shape
    h, nbl = w.spacing, w.nbl
    cells = [(nz - 1 - 4.3, 4.6, 3.7), (3.4, ny - 1 - 3.8, nx - 1 - 4.2)]
    pos = [((cz - nbl[0]) * h[0], (cy - nbl[2]) * h[1], (cx - nbl[4]) * h[2]) for cz, cy, cx in cells]
    src = np.concatenate([np.array(pos), w.src_pos])
    return dataclasses.replace(w, src_pos=src, f_peak=25.0, t0=0.02)


def face_slabs(shape, r):
    """Index tuples of the r outermost node layers of each face."""
    out = []
    for a in range(len(shape)):
        for side in (slice(0, r), slice(shape[a] - r, shape[a])):
            idx = [slice(None)] * len(shape)
            idx[a] = side
            out.append(tuple(idx))
    return out


def assert_faces_driven(p, r):
    """Each face's r outermost node layers carry a sizeable part of the field."""
    peak = np.abs(p).max()
    for idx in face_slabs(p.shape, r):
        assert np.abs(p[idx]).max() > 1e-3 * peak, idx


def assert_face_parity(p_gpu, p_ref, r):
    """Element-wise bar on each face slab against that slab's own peak (the field
    there is far smaller than in the interior behind the absorbing layers)."""
    for k, idx in enumerate(face_slabs(p_ref.shape, r)):
        assert_parity(p_gpu[idx], p_ref[idx], "face slab %d" % k, tol=FACE_TOL, max_tol=FACE_TOL)


def test_3d_layered_full_grid_faces(cuda_device):
    """Full 256^3 grid of the order-8 workload, 120 steps with sources next to every
    face: every node of the field (faces, layers, ragged tiles included) and every
    receiver sample within the bars."""
    w = face_sources(workloads.make("3d_layered_256", n_steps=120))
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    s_gpu, p_gpu = run_gpu(w, wavelet=wav, expect_variant=api.SW_STENCIL_TMA)
    s_ref, p_ref = run_oracle(w, wavelet=wav)
    assert_faces_driven(p_ref, w.order // 2)
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")
    assert_face_parity(p_gpu, p_ref, w.order // 2)


def test_3d_layered_reduced_grid_long(cuda_device):
    w = workloads.make("3d_layered_256", shape=(64, 72, 80), n_steps=400)
    s_gpu, p_gpu = run_gpu(w)
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")


def test_3d_variable_density_reduced_grid(cuda_device):
    w = workloads.make("3d_vd_512x512x384", shape=(72, 80, 96), n_steps=300)
    s_gpu, p_gpu = run_gpu(w)
    s_ref, p_ref = run_oracle(w)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")


def test_3d_variable_density_full_grid_faces(cuda_device):
    """Full 384 x 512 x 512 grid of the order-16 variable-density workload, 50
    steps with sources next to every face (the wave crosses the 8-node ghost
    reach of each face and enters every layer), element-wise."""
    w = face_sources(workloads.make("3d_vd_512x512x384", n_steps=50))
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    s_gpu, p_gpu = run_gpu(w, wavelet=wav, expect_variant=api.SW_STENCIL_TMA)
    s_ref, p_ref = run_oracle(w, wavelet=wav)
    assert_faces_driven(p_ref, w.order // 2)
    assert_parity(s_gpu, s_ref, "seismogram")
    assert_parity(p_gpu, p_ref, "field")
    assert_face_parity(p_gpu, p_ref, w.order // 2)


def test_full_length_prefix_and_invariances(cuda_device):
    """Full 2000-step 3D run: its first rows match the oracle's short run; shifting the
    wavelet by m samples shifts the trace by m rows exactly; doubling it doubles the trace
    up to FP32 rounding noise."""
    w = workloads.make("3d_layered_256")
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    s_full, _ = run_gpu(w, wavelet=wav, final=False)
    k = 40
    s_ref, _ = run_oracle(w, n_steps=k)
    assert np.abs(s_ref).max() > 0
    assert_parity(s_full[:k], s_ref, "seismogram prefix")
    m = 25
    wav_shift = np.concatenate([np.zeros(m, np.float32), wav[:-m]])
    s_shift, _ = run_gpu(w, wavelet=wav_shift, final=False)
    assert np.array_equal(s_shift[m:], s_full[:-m])
    assert not np.any(s_shift[:m])
    # Scaling by 2 is exact in FP32 only while no value is subnormal; the far
    # leading edge of the wavefield is, and from there on the two runs round
    # independently, so the difference measures the FP32 rounding noise.
    s_double, _ = run_gpu(w, wavelet=2.0 * wav, final=False)
    assert_parity(s_double, 2.0 * s_full, "seismogram")
    assert np.all(np.isfinite(s_full)) and np.abs(s_full).max() > 0


def test_zero_steps_and_no_sources(cuda_device):
    w = small_case(2, 8, False, n_steps=10)
    s, p = run_gpu(w, n_steps=0)
    assert s.shape == (0, len(w.rec_pos)) and not np.any(p)
    w.src_pos = np.zeros((0, 2))
    s, p = run_gpu(w, n_steps=10)
    assert not np.any(s) and not np.any(p)


def test_error_statuses(cuda_device):
    import torch
    w = small_case(2, 8, False, n_steps=10)
    g = api.sw_create_grid(2, w.shape, w.spacing, 8, w.nbl, w.bc, 0.0, 3, 10.0)  # dt far too large
    with pytest.raises(api.SimwaveError) as e:
        api.sw_forward(g, 1)
    assert e.value.status == api.SW_ESTATE
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_model(g, torch.from_numpy(w.velocity))
    assert e.value.status == api.SW_ECFL
    g.close()
    g = api.sw_create_grid(2, w.shape, w.spacing, 8, w.nbl, w.bc, 0.0, 3, 0.0)
    api.sw_set_model(g, torch.from_numpy(w.velocity))
    assert 0 < api.sw_get_dt(g) < 1e-2
    bad = np.array([[3.5 * w.spacing[0] - w.spacing[0] * 5, 100.0]])
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_acquisition(g, bad, w.rec_pos, np.zeros(10, np.float32), window_radius=4)
    assert e.value.status == api.SW_EINVAL
    vel_bad = w.velocity.copy()
    vel_bad[3, 4] = -1.0
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_model(g, torch.from_numpy(vel_bad))
    assert e.value.status == api.SW_EINVAL
    g.close()
    with pytest.raises(api.SimwaveError) as e:
        api.sw_create_grid(2, w.shape, w.spacing, 7, w.nbl, w.bc, 0.0, 3, 0.0)
    assert e.value.status == api.SW_EINVAL
    # variants that exist for one dimension only
    g = api.sw_create_grid(2, w.shape, w.spacing, 8, w.nbl, w.bc, 0.0, 3, 0.0)
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_stencil_variant(g, api.SW_STENCIL_TMA)
    assert e.value.status == api.SW_EINVAL
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_stencil_variant(g, 7)
    assert e.value.status == api.SW_EINVAL
    g.close()
    w3 = small_case(3, 8, False, n_steps=10)
    g = api.sw_create_grid(3, w3.shape, w3.spacing, 8, w3.nbl, w3.bc, 0.0, 3, 0.0)
    with pytest.raises(api.SimwaveError) as e:
        api.sw_set_stencil_variant(g, api.SW_STENCIL_CLUSTER)
    assert e.value.status == api.SW_EINVAL
    g.close()


def test_stalled_pipeline_reports_timeout(cuda_device):
    """Failure path without a fault: a pipeline whose copies are never issued
    runs every bounded mbarrier wait out; sw_forward returns SW_ETIMEOUT, and
    the same grid then runs normally and matches the oracle."""
    w = small_case(3, 8, False, seed=11, n_steps=20)
    import torch
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        assert api.sw_get_stencil_variant(g) == api.SW_STENCIL_TMA
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        seis = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_set_pipeline_test(g, True, 1_000_000)  # 1 ms per wait
        with pytest.raises(api.SimwaveError) as e:
            api.sw_forward(g, 3, seis)
        assert e.value.status == api.SW_ETIMEOUT
        assert "bounded wait" in api.sw_last_error()
        api.sw_set_pipeline_test(g, False, 0)
        api.sw_forward(g, w.n_steps, seis)
        s_ref, _ = run_oracle(w)
        assert_parity(seis.cpu().numpy(), s_ref, "seismogram")
    finally:
        g.close()


@pytest.mark.parametrize("ndim", [2, 3])
def test_repeated_forwards_replay_identically(cuda_device, ndim):
    """The second sw_forward with an unchanged configuration captures the time
    loop as a CUDA graph and later calls replay it: all three runs give the same
    seismogram bit for bit, and it matches the oracle; a changed step count
    runs directly again."""
    import torch
    w = small_case(ndim, 8, False, seed=21, n_steps=40)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        runs = []
        for _ in range(3):
            seis = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device=dev)
            api.sw_forward(g, w.n_steps, seis)
            runs.append(seis.cpu().numpy())
        assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])
        s_ref, _ = run_oracle(w)
        assert_parity(runs[2], s_ref)
        short = torch.zeros((w.n_steps // 2, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_forward(g, w.n_steps // 2, short)
        assert np.array_equal(short.cpu().numpy(), runs[0][: w.n_steps // 2])
    finally:
        g.close()


@pytest.mark.parametrize("ndim", [2, 3])
def test_snapshots_follow_the_saving_stride(cuda_device, ndim):
    """Frame k holds p after (k+1) * stride steps: it equals the final field of a
    run of that length (same kernels, bit for bit) and the oracle's."""
    import torch
    w = small_case(ndim, 8, False, seed=31, n_steps=37)
    dev = torch.device("cuda:0")
    stride, frames = 5, 6
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        snaps = torch.full((frames,) + tuple(w.shape), -1.0, dtype=torch.float32, device=dev)
        seis = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_set_saving(g, stride, snaps, frames)
        api.sw_forward(g, w.n_steps, seis)
        api.sw_set_saving(g, 0)
        snaps = snaps.cpu().numpy()
        for k in (0, 3, frames - 1):
            fin = torch.zeros(w.shape, dtype=torch.float32, device=dev)
            api.sw_forward(g, (k + 1) * stride, seis[: (k + 1) * stride], fin)
            assert np.array_equal(snaps[k], fin.cpu().numpy())
        _, p_ref = run_oracle(w, n_steps=4 * stride)
        assert_parity(snaps[3], p_ref, "seismogram")
        with pytest.raises(api.SimwaveError):
            api.sw_set_saving(g, 2, None, 3)
    finally:
        g.close()
