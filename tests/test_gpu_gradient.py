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


@pytest.mark.parametrize("ndim", [2, 3])
def test_every_level_kept_is_the_recomputed_gradient(cuda_device, ndim):
    """K >= n_steps: the forward run writes every level into the segment
    buffers and the sweep recomputes nothing.  The levels are the ones a
    recomputation from exact FP32 checkpoints gives (the same kernels on the
    same inputs), so the misfit is the same bits and the gradient differs
    only by the order of the Neumann correction's atomic sums (run to run);
    a 16-bit format does not apply there (nothing is stored rounded)."""
    n = 37
    w, wav, obs, _ = _setup(ndim, 8, n, seed=11 + ndim)
    J_all, g_all = _gpu_gradient(w, wav, obs, n, n)
    J_auto, g_auto = _gpu_gradient(w, wav, obs, n, 0)  # small grid: every level fits
    J_k, g_k = _gpu_gradient(w, wav, obs, n, 6)
    J_i16, g_i16 = _gpu_gradient(w, wav, obs, n, n + 5, api.SW_CKPT_I16)
    assert np.abs(g_all).max() > 0
    assert J_all == J_k == J_auto == J_i16
    assert rel_l2(g_k, g_all) <= 1e-6
    assert rel_l2(g_auto, g_all) <= 1e-6
    assert rel_l2(g_i16, g_all) <= 1e-6


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
        # every level kept (no recomputation): the same misfit, the gradient
        # up to the order of atomic sums
        gv_all = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        gr_all = np.zeros(w.shape, np.float32)
        J_all = api.sw_gradient(g, n, torch.from_numpy(obs).to(dev), gv_all, n, grad_rho=gr_all)
        assert J_all == J
        assert rel_l2(gv_all.cpu().numpy(), gv) <= 1e-6
        assert rel_l2(gr_all, gr) <= 1e-6
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


@pytest.mark.parametrize("density,fmt", [(False, api.SW_CKPT_FP32), (True, api.SW_CKPT_FP32),
                                         (False, api.SW_CKPT_BF16)])
def test_gradient_over_shots_is_the_sum_of_the_shots(cuda_device, density, fmt):
    """sw_gradient_shots over three shots (two sources each) equals the sum of
    three sw_gradient calls, matches the sum of the FP64 oracle's per-shot
    gradients, and leaves the acquisition's own sources in place."""
    import torch
    from paper_2201_05278_b300 import fwi
    n = 50
    w = small_case(3, 8, density, seed=71, n_steps=n)
    wav = np.asarray(oracle.ricker_samples(w.f_peak, w.dt, n, t0=w.t0), dtype=np.float32)
    rng = np.random.default_rng(12)
    v_true = w.velocity.astype(np.float64) * (1.0 + 0.03 * rng.standard_normal(w.shape))
    r_true = None if not density else w.density.astype(np.float64) * (1.0 + 0.05 * rng.standard_normal(w.shape))
    h = np.asarray(w.spacing)
    shots = np.stack([w.src_pos + np.array([1.3, -2.1, 2.7]) * h * k for k in range(3)])  # [3][2][3]
    kw = dict(rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc, damp_alpha=w.damp_alpha,
              damp_degree=w.damp_degree, window_radius=w.window_radius)
    obs = np.stack([oracle.forward(3, w.shape, w.spacing, w.order, v_true, w.dt, n, src_pos=[tuple(p) for p in s],
                                   wavelet=wav.astype(np.float64), rho=r_true, **kw)[0] for s in shots])
    obs = obs.astype(np.float32)
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev),
                         None if not density else torch.from_numpy(w.density).to(dev))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        before = torch.zeros((n, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_forward(g, n, before)
        gv = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        gr = torch.zeros(w.shape, dtype=torch.float32, device=dev) if density else None
        obs_d = torch.from_numpy(obs).to(dev)
        J = api.sw_gradient_shots(g, shots, n, obs_d, gv, 9, fmt, grad_rho=gr)
        after = torch.zeros_like(before)
        api.sw_forward(g, n, after)
        assert torch.equal(before, after)
        # the same through the shot-partition layer (no process group: every shot here)
        out = fwi.misfit_gradient(g, shots, obs_d, n, 9, fmt, density=density)
        assert out[0] == pytest.approx(J, rel=1e-9)  # atomic sums: equal up to their order
        assert rel_l2(out[1].cpu().numpy(), gv.cpu().numpy()) <= 1e-6
        # every level kept (one segment of all n steps; the levels of each
        # shot overwrite the previous shot's): the sums of exact levels, so
        # those of FP32 checkpoints
        gk = torch.zeros_like(gv)
        grk = torch.zeros_like(gv) if density else None
        Jk = api.sw_gradient_shots(g, shots, n, obs_d, gk, n, fmt, grad_rho=grk)
        assert Jk == pytest.approx(J, rel=1e-9)
        if fmt == api.SW_CKPT_FP32:
            assert rel_l2(gk.cpu().numpy(), gv.cpu().numpy()) <= 1e-6
            if density:
                assert rel_l2(grk.cpu().numpy(), gr.cpu().numpy()) <= 1e-6
        # shot by shot
        J1, gv1 = 0.0, torch.zeros_like(gv)
        gr1 = torch.zeros_like(gv) if density else None
        for k in range(3):
            api.sw_set_acquisition(g, shots[k], w.rec_pos, wav, window_radius=w.window_radius)
            tv = torch.zeros_like(gv)
            tr = torch.zeros_like(gv) if density else None
            J1 += api.sw_gradient(g, n, obs_d[k], tv, 9, fmt, grad_rho=tr)
            gv1 += tv
            if density:
                gr1 += tr
    finally:
        g.close()
    assert J == pytest.approx(J1, rel=1e-6)
    assert rel_l2(gv.cpu().numpy(), gv1.cpu().numpy()) <= 1e-6
    if density:
        assert rel_l2(gr.cpu().numpy(), gr1.cpu().numpy()) <= 1e-6
    if fmt == api.SW_CKPT_FP32:
        J_ref, gv_ref, gr_ref = 0.0, 0.0, 0.0
        for k in range(3):
            pb = A.make_problem(3, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                                src_pos=[tuple(p) for p in shots[k]],
                                rho=None if not density else w.density.astype(np.float64), **kw)
            j, a, b, _ = A.adjoint_gradient_full(pb, wav.astype(np.float64), obs[k].astype(np.float64), n)
            J_ref, gv_ref, gr_ref = J_ref + j, gv_ref + a, gr_ref + (b if density else 0.0)
        assert J == pytest.approx(J_ref, rel=1e-4)
        assert rel_l2(gv.cpu().numpy(), gv_ref) <= GRAD_TOL
        if density:
            assert rel_l2(gr.cpu().numpy(), gr_ref) <= GRAD_TOL


def test_gradient_over_shots_rejects_bad_shots(cuda_device):
    import torch
    w, wav, obs, _ = _setup(3, 8, 20, seed=5)
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    try:
        api.sw_set_model(g, np.ascontiguousarray(w.velocity, np.float32))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        gv = torch.zeros(w.shape, dtype=torch.float32, device="cuda:0")
        bad = np.stack([w.src_pos, w.src_pos + 1e6])  # the second shot's windows leave the grid
        with pytest.raises(api.SimwaveError) as e:
            api.sw_gradient_shots(g, bad, 20, np.stack([obs, obs]), gv)
        assert e.value.status == api.SW_EINVAL
        with pytest.raises(ValueError):
            api.sw_gradient_shots(g, np.stack([w.src_pos] * 2), 20, obs, gv)  # observed for one shot only
    finally:
        g.close()


# The misfit-gradient workload (256^3, 1500 steps, checkpoints every 10
# steps) reduced to 96^3 and 200 steps (20 checkpoints), against the FP64
# adjoint oracle.  Bars: FP32 checkpoints carry only the FP32 forward and
# adjoint (GRAD_TOL); the 16-bit formats add the rounding of the states the
# recomputed segments start from.  The 1e-2 bar for compressed snapshots is
# met by FP16 and the row-scaled 16-bit fixed point; BF16 (8 mantissa bits)
# is reported, with a loose bound that only catches a broken path.
REDUCED_FWI_TOL = {api.SW_CKPT_FP32: GRAD_TOL, api.SW_CKPT_I16: 1e-2, api.SW_CKPT_FP16: 1e-2,
                   api.SW_CKPT_BF16: 0.3}


def test_checkpoint_formats_on_the_reduced_fwi_workload(cuda_device):
    import json
    import os
    import torch
    from paper_2201_05278_b300 import workloads
    c = workloads.fwi_gradient_256(n_steps=200, shape=(96, 96, 96))
    w = c.base
    n = w.n_steps
    dev = torch.device("cuda:0")
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, n)
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    grads, Js = {}, {}
    try:
        api.sw_set_model(g, torch.from_numpy(c.v_true).to(dev))
        api.sw_set_acquisition(g, c.shots[:1], w.rec_pos, wav, window_radius=w.window_radius)
        obs = torch.zeros((n, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_forward(g, n, obs)
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        for fmt in REDUCED_FWI_TOL:
            gv = torch.zeros(w.shape, dtype=torch.float32, device=dev)
            Js[fmt] = api.sw_gradient(g, n, obs, gv, c.checkpoint_every, fmt)
            grads[fmt] = gv.cpu().numpy()
        obs = obs.cpu().numpy()
    finally:
        g.close()
    pb = A.make_problem(3, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                        src_pos=[tuple(c.shots[0])], rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc,
                        damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)
    J_ref, g_ref, _ = A.adjoint_gradient(pb, np.asarray(wav, np.float64), obs.astype(np.float64), n)
    errs = {fmt: rel_l2(grads[fmt], g_ref) for fmt in grads}
    names = {api.SW_CKPT_FP32: "fp32", api.SW_CKPT_BF16: "bf16", api.SW_CKPT_FP16: "fp16", api.SW_CKPT_I16: "i16"}
    print("reduced fwi workload, gradient rel-L2 against the FP64 oracle: " +
          ", ".join("%s %.3e" % (names[f], e) for f, e in errs.items()))
    log = os.environ.get("PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"test": "reduced_fwi_checkpoint_formats",
                                "rel_l2": {names[k]: v for k, v in errs.items()}}) + "\n")
    for fmt, e in errs.items():
        assert Js[fmt] == pytest.approx(J_ref, rel=1e-4)
        assert e <= REDUCED_FWI_TOL[fmt], (names[fmt], e)
