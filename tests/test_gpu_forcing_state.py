"""GPU tests of distributed forcing, initial levels and snapshot-based resume.

- Standing waves: with p[0] = p[-1] = an exact discrete eigenmode of the
  Eq. 9 Laplacian (sine modes under Dirichlet faces, cosine modes under
  Neumann faces), the CUDA path must follow the closed-form solution of the
  two-level recurrence (Eq. 7), with both 3D kernels and the 2D kernel.
- Manufactured solutions (Sec. 2.5, Eq. 14-15): the distributed forcing on
  the GPU reproduces the oracle's field and second-order convergence in time;
  the variable-density forcing matches the oracle too.
- Random forcing on the mixed-face test grids, against the oracle.
- Resume: restarting from two saved levels continues the run.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2201_05278_b300 import api
from tests import analytic
from tests.harness import FP32_SEIS_TOL, assert_parity, rel_l2, run_oracle
from tests.test_gpu_parity import small_case
from tests.test_oracle_solver import _mode

pytestmark = pytest.mark.gpu


def _grid(w, variant=None):
    import torch
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    api.sw_set_model(g, torch.from_numpy(np.ascontiguousarray(w.velocity, np.float32)).cuda(),
                     None if w.density is None else torch.from_numpy(np.ascontiguousarray(w.density, np.float32)).cuda())
    if variant is not None:
        api.sw_set_stencil_variant(g, variant)
    return g


def _final(g, n_steps, n_rec=0):
    import torch
    seis = torch.zeros((n_steps, n_rec), dtype=torch.float32, device="cuda:0")
    fin = torch.zeros(g.shape, dtype=torch.float32, device="cuda:0")
    api.sw_forward(g, n_steps, seis if n_rec else None, fin)
    return seis.cpu().numpy(), fin.cpu().numpy()


class _Plain:
    """A bare grid description (no sources, no damping) for the closed-form cases."""

    def __init__(self, ndim, shape, spacing, order, bc, vel, dt, density=None):
        self.ndim, self.shape, self.spacing, self.order = ndim, tuple(shape), tuple(spacing), order
        self.nbl, self.bc, self.damp_alpha, self.damp_degree, self.dt = [0] * (2 * ndim), bc, 0.0, 3, dt
        self.velocity, self.density = vel, density


@pytest.mark.parametrize("ndim,order,variant", [(2, 4, None), (2, 16, None), (3, 8, api.SW_STENCIL_PLAIN),
                                                (3, 8, api.SW_STENCIL_TMA), (3, 20, api.SW_STENCIL_TMA)])
@pytest.mark.parametrize("kind", ["d", "n"])
def test_standing_mode_follows_the_closed_form(cuda_device, ndim, order, variant, kind):
    r = order // 2
    shape = (r + 19, r + 15, r + 27) if ndim == 3 else (r + 29, r + 37)
    spacing = (3.0, 4.0, 5.0) if ndim == 3 else (3.0, 5.0)
    m = (2, 1, 3) if ndim == 3 else (2, 3)
    mode, lam = _mode(shape, spacing, [kind] * ndim, m, order)
    c, n_steps = 700.0, 150
    dt = 0.3 * min(spacing) / c
    bc = ["null_dirichlet" if kind == "d" else "null_neumann"] * (2 * ndim)
    w = _Plain(ndim, shape, spacing, order, bc, np.full(shape, c, np.float32), dt)
    g = _grid(w, variant)
    try:
        api.sw_set_acquisition(g, np.zeros((0, ndim)), np.zeros((0, ndim)), np.zeros(1, np.float32))
        api.sw_set_initial_state(g, mode.astype(np.float32), mode.astype(np.float32))
        _, p = _final(g, n_steps)
    finally:
        g.close()
    # a_{n+1} = (2 + kappa lam) a_n - a_{n-1}, a_0 = a_{-1} = 1
    kappa = (c * dt) ** 2
    b = -(2.0 + kappa * lam)
    disc = complex(b * b - 4.0)
    mu1, mu2 = (-b + disc ** 0.5) / 2, (-b - disc ** 0.5) / 2
    B = (1 - 1 / mu1) / (1 / mu2 - 1 / mu1)
    amp = ((1 - B) * mu1 ** n_steps + B * mu2 ** n_steps).real
    assert np.abs(p - amp * mode).max() <= 1e-4 * np.abs(mode).max()


def _mms_gpu(order, h, dt, t_end, density, c=2000.0, L=440.0):
    """(normalised GPU - oracle difference, normalised GPU error, normalised oracle error).

    Normalised by the spatial shape of the solution (|T(t)| <= 1), as the
    oracle's own convergence tests do: u*(t_N) itself can vanish."""
    n = int(round(L / h)) + 1
    steps = int(round(t_end / dt))
    rho, F, T, uN = analytic.mms_2d(L, c, n, n, h, dt, steps, density)
    bc = ["null_dirichlet"] * 4
    w = _Plain(2, (n, n), (h, h), order, bc, np.full((n, n), c, np.float32), dt,
               None if rho is None else rho.astype(np.float32))
    g = _grid(w)
    try:
        api.sw_set_acquisition(g, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(1, np.float32))
        api.sw_set_forcing(g, F, T)
        _, p = _final(g, steps)
    finally:
        g.close()
    _, p_ref = oracle.forward(2, (n, n), (h, h), order, np.full((n, n), c), dt, steps, nbl=[0] * 4, bc=bc,
                              rho=rho, force_fields=F, force_sigs=T)
    norm = np.linalg.norm(analytic.mms_2d(L, c, n, n, h, dt, 0, None)[1][0]) * c * c
    return np.linalg.norm(p - p_ref) / norm, np.linalg.norm(p - uN) / norm, np.linalg.norm(p_ref - uN) / norm


def test_manufactured_solution_second_order_in_time(cuda_device):
    errs = []
    for dt in (1.6e-3, 8e-4, 4e-4):
        d, e, e_ref = _mms_gpu(16, 11.0, dt, 0.1, None)
        # FP32 rounding (about 2e-8 of the field per step) stays well below the
        # discretisation error: 0.5% of it at 1.6e-3, 4% at 4e-4 (250 steps)
        assert d <= 0.1 * e_ref
        assert e == pytest.approx(e_ref, rel=0.1)
        errs.append(e)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < r < 2.1 for r in rates), (errs, rates)


def test_manufactured_solution_variable_density(cuda_device):
    d, e, e_ref = _mms_gpu(4, 11.0, 8e-4, 0.1, "cos")
    assert d <= 1e-2 * e_ref
    assert e == pytest.approx(e_ref, rel=1e-2)


@pytest.mark.parametrize("ndim,variant", [(2, None), (3, api.SW_STENCIL_PLAIN), (3, api.SW_STENCIL_TMA)])
def test_random_forcing_against_the_oracle(cuda_device, ndim, variant):
    """Forcing plus point sources on damped grids with mixed face conditions."""
    w = small_case(ndim, 8, False, seed=41, n_steps=50)
    rng = np.random.default_rng(7)
    F = rng.standard_normal((2,) + tuple(w.shape)).astype(np.float32)
    T = (0.2 * rng.standard_normal((2, w.n_steps))).astype(np.float32)
    g = _grid(w, variant)
    try:
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        api.sw_set_forcing(g, F, T)
        s, p = _final(g, w.n_steps, len(w.rec_pos))
        with pytest.raises(api.SimwaveError):  # signatures shorter than the run
            _final(g, w.n_steps + 1, len(w.rec_pos))
    finally:
        g.close()
    wav = oracle.ricker_samples(w.f_peak, w.dt, w.n_steps, t0=w.t0)
    s_ref, p_ref = oracle.forward(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                                  w.n_steps, src_pos=[tuple(q) for q in w.src_pos], wavelet=wav,
                                  rec_pos=[tuple(q) for q in w.rec_pos], nbl=w.nbl, bc=w.bc,
                                  damp_alpha=w.damp_alpha, damp_degree=w.damp_degree,
                                  window_radius=w.window_radius, force_fields=F.astype(np.float64),
                                  force_sigs=T.astype(np.float64))
    assert_parity(s, s_ref, "seismogram")
    assert_parity(p, p_ref, "field")


@pytest.mark.parametrize("ndim", [2, 3])
def test_resume_from_two_saved_levels(cuda_device, ndim):
    """Run N steps; run N1 saving every step, then restart from (p[N1], p[N1-1])
    with the wavelet shifted by N1: the rest of the run is the same."""
    import torch
    w = small_case(ndim, 8, False, seed=43, n_steps=48)
    n1 = 20
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    g = _grid(w)
    try:
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
        s_full, p_full = _final(g, w.n_steps, len(w.rec_pos))
        snaps = torch.zeros((n1,) + tuple(w.shape), dtype=torch.float32, device="cuda:0")
        api.sw_set_saving(g, 1, snaps, n1)
        _final(g, n1, len(w.rec_pos))
        api.sw_set_saving(g, 0)
        api.sw_set_initial_state(g, snaps[n1 - 1], snaps[n1 - 2])
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, np.ascontiguousarray(wav[n1:]),
                               window_radius=w.window_radius)
        s_rest, p_rest = _final(g, w.n_steps - n1, len(w.rec_pos))
        with pytest.raises(api.SimwaveError):  # the gradient starts from rest
            api.sw_gradient(g, 4, torch.zeros((4, len(w.rec_pos)), device="cuda:0"),
                            torch.zeros(w.shape, device="cuda:0"))
    finally:
        g.close()
    assert rel_l2(s_rest, s_full[n1:]) <= 1e-6
    assert rel_l2(p_rest, p_full) <= 1e-6
    _, p_ref = run_oracle(w)
    assert_parity(p_rest, p_ref, "field")
