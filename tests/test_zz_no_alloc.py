"""The allocation-free forward entry point (sw_forward_noalloc) against sw_forward.

sw_forward_noalloc serves callers that cannot call cudaMalloc (device memory
owned by a fixed-budget pool or framework allocator, or loops that cannot
afford cudaMalloc's device-wide synchronisation): it keeps its wavefields and
tables in one static device array instead.  These tests call it through the
C ABI twice in a row (the array keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared) and
compare with the handle-based sw_forward and with the FP64 oracle, within the
parity tolerance.  The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2201_05278_b300 import api
from tests.harness import FP32_SEIS_TOL, assert_parity, rel_l2, run_gpu, run_oracle
from tests.test_gpu_parity import small_case

pytestmark = pytest.mark.gpu


def _noalloc(w, n_steps):
    import torch
    dev = torch.device("cuda:0")
    vel = torch.from_numpy(np.ascontiguousarray(w.velocity, np.float32)).to(dev)
    rho = None if w.density is None else torch.from_numpy(np.ascontiguousarray(w.density, np.float32)).to(dev)
    seis = torch.full((n_steps, len(w.rec_pos)), float("nan"), dtype=torch.float32, device=dev)
    fin = torch.full(w.shape, float("nan"), dtype=torch.float32, device=dev)
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, n_steps)
    api.sw_forward_noalloc(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                           vel, rho, w.src_pos, w.rec_pos, wav, w.window_radius, n_steps, seis, fin)
    return seis.cpu().numpy(), fin.cpu().numpy()


@pytest.mark.parametrize("ndim,order,density", [(2, 8, False), (3, 8, False), (3, 16, True)])
def test_noalloc_matches_sw_forward_twice(cuda_device, ndim, order, density):
    w = small_case(ndim, order, density, seed=11 + order, n_steps=50)
    s_ref, p_ref = run_gpu(w)
    s_or, p_or = run_oracle(w)
    for _ in range(2):
        s, p = _noalloc(w, w.n_steps)
        assert np.all(np.isfinite(s)) and np.all(np.isfinite(p))
        assert_parity(s, s_ref, "seismogram")
        assert_parity(p, p_ref, "field")
        assert_parity(s, s_or, "seismogram vs oracle")
        assert_parity(p, p_or, "field vs oracle")


def _raw_call(shape, vel_ptr, n_steps=1):
    """sw_forward_noalloc through the C ABI directly (no Python-side size checks)."""
    import ctypes
    from paper_2201_05278_b300 import _lib
    nd = len(shape)
    shp = (ctypes.c_int64 * nd)(*shape)
    spc = (ctypes.c_double * nd)(*([10.0] * nd))
    nbl = (ctypes.c_int * (2 * nd))(*([0] * (2 * nd)))
    bc = (ctypes.c_int * (2 * nd))(*([api.SW_BC_DIRICHLET] * (2 * nd)))
    return _lib.load().sw_forward_noalloc(nd, shp, spc, 8, nbl, bc, 0.0, 3, 1e-3, ctypes.c_void_p(vel_ptr), None,
                                          0, None, 0, None, 0, None, 0, 4, n_steps, None, None, None)


def test_noalloc_rejects_oversized_problem(cuda_device):
    """Sizes beyond the static array are refused before any device work: a
    512^3 grid needs about three padded copies of 537 MB, and a grid past
    2^34 nodes is refused outright (no size arithmetic can wrap)."""
    import torch
    vel = torch.empty(1, dtype=torch.float32, device="cuda:0")
    assert _raw_call((512, 512, 512), vel.data_ptr()) == api.SW_EINVAL
    assert "scratch" in api.sw_last_error()
    assert _raw_call((1 << 24, 1 << 24, 1 << 12), vel.data_ptr()) == api.SW_EINVAL
    assert "too large" in api.sw_last_error()


def test_noalloc_checks_buffers(cuda_device):
    """Host memory where device memory of the current device is needed is
    refused by the library; undersized tensors by the Python binding."""
    import torch
    w = small_case(2, 8, False, seed=2, n_steps=10)
    host = np.ascontiguousarray(w.velocity, np.float32)
    assert _raw_call(w.shape, host.ctypes.data) == api.SW_EINVAL
    assert "device memory of the current device" in api.sw_last_error()
    vel = torch.from_numpy(host).cuda()
    seis = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device="cuda:0")
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    args = (w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    with pytest.raises(ValueError):
        api.sw_forward_noalloc(*args, vel[:-1], None, w.src_pos, w.rec_pos, wav, 4, w.n_steps, seis)
    with pytest.raises(ValueError):
        api.sw_forward_noalloc(*args, vel, None, w.src_pos, w.rec_pos, wav, 4, w.n_steps, seis[:-1])
    with pytest.raises(ValueError):  # one wavelet for two sources declared per source
        api.sw_forward_noalloc(*args, vel, None, w.src_pos, w.rec_pos, wav, 4, w.n_steps, seis,
                               wavelet_per_source=True)


def test_noalloc_per_source_wavelets_on_the_device(cuda_device):
    """Per-source wavelets already in device memory, against sw_forward with the same wavelets."""
    import torch
    w = small_case(3, 8, False, seed=19, n_steps=40)
    dev = torch.device("cuda:0")
    base = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    wav = np.stack([base, -0.5 * base])  # [n_src][nt]
    assert wav.shape[0] == len(w.src_pos)
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius, wavelet_per_source=True)
        s_ref = torch.zeros((w.n_steps, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_forward(g, w.n_steps, s_ref)
    finally:
        g.close()
    vel = torch.from_numpy(w.velocity).to(dev)
    wav_d = torch.from_numpy(wav).to(dev)
    for _ in range(2):
        seis = torch.full((w.n_steps, len(w.rec_pos)), float("nan"), dtype=torch.float32, device=dev)
        api.sw_forward_noalloc(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                               vel, None, w.src_pos, w.rec_pos, wav_d, w.window_radius, w.n_steps, seis,
                               wavelet_per_source=True)
        assert_parity(seis.cpu().numpy(), s_ref.cpu().numpy(), "seismogram")
