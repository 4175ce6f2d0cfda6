"""The allocation-free forward entry point (sw_forward_noalloc) against sw_forward.

sw_forward_noalloc serves callers that cannot call cudaMalloc (device memory
owned by a fixed-budget pool or framework allocator, or loops that cannot
afford cudaMalloc's device-wide synchronisation): it keeps its wavefields and
tables in one static device array instead.  These tests call it through the
C ABI twice in a row (the array keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared) and
compare with the handle-based sw_forward within the parity tolerance.  The
file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2201_05278_b300 import api
from tests.harness import FP32_SEIS_TOL, rel_l2, run_gpu
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
    for _ in range(2):
        s, p = _noalloc(w, w.n_steps)
        assert np.all(np.isfinite(s)) and np.all(np.isfinite(p))
        assert rel_l2(s, s_ref) <= FP32_SEIS_TOL
        assert rel_l2(p, p_ref) <= FP32_SEIS_TOL


def test_noalloc_rejects_oversized_problem(cuda_device):
    import torch
    shape = (512, 512, 512)  # ~3 padded copies of 537 MB: far beyond the scratch limit
    vel = torch.empty(1, dtype=torch.float32, device="cuda:0")
    with pytest.raises(api.SimwaveError) as e:
        api.sw_forward_noalloc(3, shape, (10.0, 10.0, 10.0), 8, [0] * 6, ["null_dirichlet"] * 6, 0.0, 3, 1e-3,
                               vel, None, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(1, np.float32), 4, 1)
    assert e.value.status == api.SW_EINVAL
    assert "scratch" in str(e.value)
