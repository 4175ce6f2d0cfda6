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


def test_density_gradient_needs_a_density_model(cuda_device):
    w, wav, obs, _ = _setup(2, 8, 10, seed=2)
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, np.ascontiguousarray(w.velocity, np.float32))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        with pytest.raises(api.SimwaveError) as e:
            api.sw_gradient(g, 10, obs, np.zeros(w.shape, np.float32), grad_rho=np.zeros(w.shape, np.float32))
        assert e.value.status == api.SW_EINVAL
    finally:
        g.close()


@pytest.mark.parametrize("ndim,order,variant", [(2, 8, None), (3, 8, api.SW_STENCIL_TMA),
                                                (3, 8, api.SW_STENCIL_PLAIN), (3, 4, None)])
def test_variable_density_gradients_match_oracle(cuda_device, ndim, order, variant):
    """dJ/dc and dJ/drho of the density model against the FP64 oracle."""
    import torch
    n = 50
    w = small_case(ndim, order, True, seed=60 + ndim + order, n_steps=n)
    wav = np.asarray(oracle.ricker_samples(w.f_peak, w.dt, n, t0=w.t0), dtype=np.float32)
    rng = np.random.default_rng(9)
    v_true = w.velocity.astype(np.float64) * (1.0 + 0.03 * rng.standard_normal(w.shape))
    r_true = w.density.astype(np.float64) * (1.0 + 0.05 * rng.standard_normal(w.shape))
    kw = dict(src_pos=[tuple(p) for p in w.src_pos], rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc,
              damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)
    obs, _ = oracle.forward(w.ndim, w.shape, w.spacing, w.order, v_true, w.dt, n, wavelet=wav.astype(np.float64),
                            rho=r_true, **kw)
    obs = obs.astype(np.float32)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev), torch.from_numpy(w.density).to(dev))
        if variant is not None:
            api.sw_set_stencil_variant(g, variant)
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        gv = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        gr = np.zeros(w.shape, np.float32)  # host output
        J = api.sw_gradient(g, n, torch.from_numpy(obs).to(dev), gv, 9, grad_rho=gr)
        gv = gv.cpu().numpy()
    finally:
        g.close()
    pb = A.make_problem(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                        rho=w.density.astype(np.float64), **kw)
    J_ref, gv_ref, gr_ref, _ = A.adjoint_gradient_full(pb, wav.astype(np.float64), obs.astype(np.float64), n)
    assert J == pytest.approx(J_ref, rel=1e-4)
    assert np.abs(gr_ref).max() > 0
    assert rel_l2(gv, gv_ref) <= GRAD_TOL
    assert rel_l2(gr, gr_ref) <= GRAD_TOL


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


def test_autograd_density_gradient(cuda_device):
    import torch
    from paper_2201_05278_b300 import autograd
    n = 40
    w = small_case(2, 8, True, seed=13, n_steps=n)
    wav = np.asarray(oracle.ricker_samples(w.f_peak, w.dt, n, t0=w.t0), dtype=np.float32)
    kw = dict(src_pos=[tuple(p) for p in w.src_pos], rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc,
              damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)
    obs, _ = oracle.forward(w.ndim, w.shape, w.spacing, w.order, 1.02 * w.velocity.astype(np.float64), w.dt, n,
                            wavelet=wav.astype(np.float64), rho=0.97 * w.density.astype(np.float64), **kw)
    obs = obs.astype(np.float32)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        vel = torch.from_numpy(w.velocity).to(dev).requires_grad_(True)
        rho = torch.from_numpy(w.density).to(dev).requires_grad_(True)
        api.sw_set_model(g, vel.detach(), rho.detach())
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        J = autograd.misfit(vel, g, torch.from_numpy(obs).to(dev), n, density=rho)
        J.backward()
        pb = A.make_problem(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                            rho=w.density.astype(np.float64), **kw)
        J_ref, gv_ref, gr_ref, _ = A.adjoint_gradient_full(pb, wav.astype(np.float64), obs.astype(np.float64), n)
        assert float(J.detach()) == pytest.approx(J_ref, rel=1e-4)
        assert rel_l2(vel.grad.cpu().numpy(), gv_ref) <= GRAD_TOL
        assert rel_l2(rho.grad.cpu().numpy(), gr_ref) <= GRAD_TOL
    finally:
        g.close()


# Gradient error against the FP64 oracle with 16-bit checkpoints (the
# recomputed segments start from rounded states); bounds from the mantissa
# widths (8 bits BF16, 11 bits FP16).
# BF16 at the 1e-2 bar for compressed snapshots; FP16 and the row-scaled
# fixed point well inside it (measured 3.5e-3, 3.7e-4, 7.1e-5 on this case)
CKPT_TOL = {api.SW_CKPT_BF16: 1e-2, api.SW_CKPT_FP16: 2e-3, api.SW_CKPT_I16: 5e-4}


@pytest.mark.parametrize("fmt", [api.SW_CKPT_BF16, api.SW_CKPT_FP16, api.SW_CKPT_I16])
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


@pytest.mark.parametrize("ndim", [2, 3])
def test_binomial_checkpointing_gives_the_same_gradient(cuda_device, ndim):
    """A memory budget of 1, 2 or 5 stored states (binomial schedule) gives the
    uniform scheme's misfit and gradient; BF16 checkpoints are refused there."""
    import torch
    n = 37
    w, wav, obs, _ = _setup(ndim, 8, n, seed=21)
    J0, g0 = _gpu_gradient(w, wav, obs, n, 6)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(np.ascontiguousarray(w.velocity, np.float32)).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        for budget in (1, 2, 5):
            api.sw_set_checkpoint_budget(g, budget)
            grad = torch.zeros(w.shape, dtype=torch.float32, device=dev)
            J = api.sw_gradient(g, n, torch.from_numpy(obs).to(dev), grad)
            assert J == J0
            assert rel_l2(grad.cpu().numpy(), g0) <= 1e-6
        with pytest.raises(api.SimwaveError):
            api.sw_gradient(g, n, torch.from_numpy(obs).to(dev), grad, 0, api.SW_CKPT_BF16)
        with pytest.raises(api.SimwaveError):
            api.sw_set_checkpoint_budget(g, -1)
    finally:
        g.close()
