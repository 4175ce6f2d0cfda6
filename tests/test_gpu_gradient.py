"""GPU misfit gradient (sw_gradient, adjoint-state method) against the FP64
adjoint oracle (oracle/adjoint.py, itself pinned by a dot-product test and
finite differences in tests/test_oracle_adjoint.py)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as A
from paper_2201_05278_b300 import api

from test_gpu_parity import small_case
from harness import rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 2e-3  # relative L2, FP32 forward + adjoint + imaging vs FP64


def _setup(ndim, order, n_steps, seed):
    w = small_case(ndim, order, False, seed=seed, n_steps=n_steps)
    wav = np.asarray(oracle.ricker_samples(w.f_peak, w.dt, n_steps, t0=w.t0), dtype=np.float32)
    rng = np.random.default_rng(seed + 1)
    v_true = (w.velocity * (1.0 + 0.03 * rng.standard_normal(w.velocity.shape))).astype(np.float64)
    kw = dict(src_pos=[tuple(p) for p in w.src_pos], rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc,
              damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)
    obs, _ = oracle.forward(w.ndim, w.shape, w.spacing, w.order, v_true, w.dt, n_steps,
                            wavelet=wav.astype(np.float64), **kw)
    return w, wav, obs.astype(np.float32), kw


def _gpu_gradient(w, wav, obs, n_steps, checkpoint_every=0, fmt=api.SW_CKPT_FP32):
    import torch
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(np.ascontiguousarray(w.velocity, np.float32)).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        grad = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        J = api.sw_gradient(g, n_steps, torch.from_numpy(obs).to(dev), grad, checkpoint_every, fmt)
        return J, grad.cpu().numpy()
    finally:
        g.close()


@pytest.mark.parametrize("ndim,order", [(2, 8), (3, 8), (3, 4)])
def test_gradient_matches_oracle(cuda_device, ndim, order):
    n = 60
    w, wav, obs, kw = _setup(ndim, order, n, seed=40 + ndim + order)
    J, grad = _gpu_gradient(w, wav, obs, n)
    pb = A.make_problem(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt, **kw)
    J_ref, g_ref, _ = A.adjoint_gradient(pb, wav.astype(np.float64), obs.astype(np.float64), n)
    assert J == pytest.approx(J_ref, rel=1e-4)
    assert np.abs(g_ref).max() > 0
    assert rel_l2(grad, g_ref) <= GRAD_TOL


def test_gradient_does_not_depend_on_checkpoint_interval(cuda_device):
    n = 45
    w, wav, obs, _ = _setup(3, 8, n, seed=3)
    J0, g0 = _gpu_gradient(w, wav, obs, n, 0)
    for K in (1, 7, n):
        J, gk = _gpu_gradient(w, wav, obs, n, K)
        assert J == J0
        assert rel_l2(gk, g0) <= 1e-6


def test_gradient_rejects_what_it_does_not_cover(cuda_device):
    import torch
    w = small_case(3, 8, True, seed=2, n_steps=10)
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity), torch.from_numpy(w.density))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, 10), window_radius=4)
        obs = np.zeros((10, len(w.rec_pos)), np.float32)
        grad = np.zeros(w.shape, np.float32)
        with pytest.raises(api.SimwaveError) as e:
            api.sw_gradient(g, 10, obs, grad)
        assert e.value.status == api.SW_EINVAL
    finally:
        g.close()


def test_autograd_misfit_backward_gives_the_adjoint_gradient(cuda_device):
    import torch
    from paper_2201_05278_b300 import autograd
    n = 40
    w, wav, obs, kw = _setup(3, 8, n, seed=9)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        vel = torch.from_numpy(np.ascontiguousarray(w.velocity, np.float32)).to(dev).requires_grad_(True)
        api.sw_set_model(g, vel.detach())
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        J = autograd.misfit(vel, g, torch.from_numpy(obs).to(dev), n)
        (2.0 * J).backward()
        pb = A.make_problem(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt, **kw)
        J_ref, g_ref, _ = A.adjoint_gradient(pb, wav.astype(np.float64), obs.astype(np.float64), n)
        assert float(J.detach()) == pytest.approx(J_ref, rel=1e-4)
        assert rel_l2(vel.grad.cpu().numpy(), 2.0 * g_ref) <= GRAD_TOL
    finally:
        g.close()


# Gradient error against the FP64 oracle with 16-bit checkpoints (the
# recomputed segments start from rounded states); bounds from the mantissa
# widths (8 bits BF16, 11 bits FP16).
CKPT_TOL = {api.SW_CKPT_BF16: 3e-2, api.SW_CKPT_FP16: 5e-3}


@pytest.mark.parametrize("fmt", [api.SW_CKPT_BF16, api.SW_CKPT_FP16])
def test_gradient_with_16_bit_checkpoints(cuda_device, fmt):
    n = 60
    w, wav, obs, kw = _setup(3, 8, n, seed=12)
    J, grad = _gpu_gradient(w, wav, obs, n, 8, fmt)
    pb = A.make_problem(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt, **kw)
    J_ref, g_ref, _ = A.adjoint_gradient(pb, wav.astype(np.float64), obs.astype(np.float64), n)
    err = rel_l2(grad, g_ref)
    print("checkpoint format %d: gradient rel-L2 error %.3e against the FP64 oracle" % (fmt, err))
    assert J == pytest.approx(J_ref, rel=1e-4)  # the forward pass itself is not rounded
    assert err <= CKPT_TOL[fmt]
