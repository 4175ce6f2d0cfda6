"""Pins of the FP64 adjoint oracle (oracle/adjoint.py):

- its own forward equals oracle.c's forward (the C loop of Eq. 7);
- laplacian_t is the transpose of the matrix of laplacian on tiny grids with
  every face condition (brute force);
- dot-product test: <F s, r> = <s, F^T r> for the linear wavelet-to-seismogram
  map F (forward from oracle.c, adjoint from the numpy sweep);
- the misfit gradient w.r.t. velocity agrees with centred finite differences
  of the misfit computed by oracle.c.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as A

BC3 = ["null_neumann", "null_dirichlet", "null_dirichlet", "none", "null_neumann", "null_dirichlet"]
BC2 = ["null_neumann", "null_dirichlet", "none", "null_neumann"]


def _case(ndim, seed=0, n_steps=40):
    rng = np.random.default_rng(seed)
    if ndim == 3:
        shape, spacing, nbl, bc = (14, 13, 15), (9.0, 8.0, 10.0), [0, 3, 2, 3, 3, 2], BC3
    else:
        shape, spacing, nbl, bc = (24, 27), (7.0, 9.0), [0, 5, 4, 6], BC2
    vel = 1800.0 + 700.0 * rng.random(shape)
    dt = 0.3 * min(spacing) / vel.max()
    phys = [(shape[a] - nbl[2 * a] - nbl[2 * a + 1] - 1) * spacing[a] for a in range(ndim)]
    src = [[0.37 * p for p in phys]]
    rec = [[0.6 * p for p in phys], [0.25 * p + 1.3 for p in phys], [spacing[0]] + [0.5 * p for p in phys[1:]]]
    kw = dict(src_pos=src, rec_pos=rec, nbl=nbl, bc=bc, damp_alpha=30.0 / max(nbl) ** 3, damp_degree=3,
              window_radius=3)
    wav = oracle.ricker_samples(30.0, dt, n_steps, t0=1.0 / 30.0)
    return shape, spacing, vel, dt, kw, wav, n_steps


@pytest.mark.parametrize("ndim", [2, 3])
def test_numpy_forward_equals_oracle_c(ndim):
    shape, spacing, vel, dt, kw, wav, n = _case(ndim)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, **kw)
    states, seis = A.forward_states(pb, wav, n)
    seis_c, p_c = oracle.forward(ndim, shape, spacing, 6, vel, dt, n, wavelet=np.asarray(wav), **kw)
    assert np.abs(seis - seis_c).max() <= 1e-12 * np.abs(seis_c).max()
    assert np.abs(states[-1] - p_c).max() <= 1e-12 * np.abs(p_c).max()


@pytest.mark.parametrize("ndim", [2, 3])
def test_laplacian_t_is_the_matrix_transpose(ndim):
    if ndim == 3:
        shape, spacing, bc = (9, 10, 11), (7.0, 8.0, 9.0), BC3
    else:
        shape, spacing, bc = (11, 13), (7.0, 9.0), BC2
    pb = A.make_problem(ndim, shape, spacing, 6, np.full(shape, 2000.0), 1e-3, bc=bc)
    n = int(np.prod(shape))
    L = np.zeros((n, n))
    LT = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        L[:, i] = A.laplacian(e.reshape(shape), pb).ravel()
        LT[:, i] = A.laplacian_t(e.reshape(shape), pb).ravel()
    keep = np.ones(shape, bool)  # Z: Dirichlet face nodes are held at zero on both sides
    for ax in range(ndim):
        for side, kind in enumerate(pb.bc[ax]):
            if kind == oracle.BC_DIRICHLET:
                idx = [slice(None)] * ndim
                idx[ax] = 0 if side == 0 else shape[ax] - 1
                keep[tuple(idx)] = False
    k = keep.ravel()
    assert np.abs(L.T[np.ix_(k, k)] - LT[np.ix_(k, k)]).max() <= 1e-15 * np.abs(L).max()
    assert np.abs(L - LT).max() > 1e-3 * np.abs(L).max()  # the Neumann faces do make L non-symmetric


@pytest.mark.parametrize("ndim", [2, 3])
def test_dot_product(ndim):
    shape, spacing, vel, dt, kw, _, n = _case(ndim, seed=5)
    rng = np.random.default_rng(11)
    s = rng.standard_normal(n)
    r = rng.standard_normal((n, len(kw["rec_pos"])))
    seis_c, _ = oracle.forward(ndim, shape, spacing, 6, vel, dt, n, wavelet=s, **kw)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, **kw)
    _, adj = A.backward(pb, r, n)
    lhs = float(np.sum(seis_c * r))
    rhs = float(np.sum(s * adj[0]))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-300)


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_matches_finite_differences(ndim):
    shape, spacing, vel, dt, kw, wav, n = _case(ndim, seed=7)
    rng = np.random.default_rng(3)
    vel_true = vel * (1.0 + 0.02 * rng.standard_normal(shape))
    obs, _ = oracle.forward(ndim, shape, spacing, 6, vel_true, dt, n, wavelet=np.asarray(wav), **kw)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, **kw)
    J, g, _ = A.adjoint_gradient(pb, wav, obs, n)
    assert J > 0
    dv = rng.standard_normal(shape)

    def misfit(v):
        d, _ = oracle.forward(ndim, shape, spacing, 6, v, dt, n, wavelet=np.asarray(wav), **kw)
        return 0.5 * float(np.sum((d - obs) ** 2))

    eps = 1e-3
    fd = (misfit(vel + eps * dv) - misfit(vel - eps * dv)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g * dv)), rel=1e-6)


# ---- variable density (Eq. 5 with the Eq. 10 term) --------------------------

def _rho(shape, seed):
    rng = np.random.default_rng(seed)
    return 1500.0 + 1200.0 * rng.random(shape)


@pytest.mark.parametrize("ndim", [2, 3])
def test_numpy_forward_equals_oracle_c_variable_density(ndim):
    shape, spacing, vel, dt, kw, wav, n = _case(ndim)
    rho = _rho(shape, 1)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, rho=rho, **kw)
    states, seis = A.forward_states(pb, wav, n)
    seis_c, p_c = oracle.forward(ndim, shape, spacing, 6, vel, dt, n, wavelet=np.asarray(wav), rho=rho, **kw)
    assert np.abs(seis - seis_c).max() <= 1e-12 * np.abs(seis_c).max()
    assert np.abs(states[-1] - p_c).max() <= 1e-12 * np.abs(p_c).max()


@pytest.mark.parametrize("even", [False, True])
@pytest.mark.parametrize("ndim", [2, 3])
def test_first_derivative_transpose_is_the_matrix_transpose(ndim, even):
    if ndim == 3:
        shape, spacing, bc = (9, 10, 11), (7.0, 8.0, 9.0), BC3
    else:
        shape, spacing, bc = (11, 13), (7.0, 9.0), BC2
    pb = A.make_problem(ndim, shape, spacing, 6, np.full(shape, 2000.0), 1e-3, bc=bc)
    n = int(np.prod(shape))
    for ax in range(ndim):
        D = np.zeros((n, n))
        DT = np.zeros((n, n))
        for i in range(n):
            e = np.zeros(n)
            e[i] = 1.0
            D[:, i] = A.first_deriv(e.reshape(shape), pb, ax, even).ravel()
            DT[:, i] = A.first_deriv_t(e.reshape(shape), pb, ax, even).ravel()
        assert np.abs(D.T - DT).max() <= 1e-15 * np.abs(D).max()


@pytest.mark.parametrize("ndim", [2, 3])
def test_variable_density_operator_transpose(ndim):
    if ndim == 3:
        shape, spacing, bc = (9, 10, 11), (7.0, 8.0, 9.0), BC3
    else:
        shape, spacing, bc = (11, 13), (7.0, 9.0), BC2
    pb = A.make_problem(ndim, shape, spacing, 6, np.full(shape, 2000.0), 1e-3, bc=bc, rho=_rho(shape, 2))
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    MT = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = A.operator(e.reshape(shape), pb).ravel()
        MT[:, i] = A.operator_t(e.reshape(shape), pb).ravel()
    keep = np.ones(shape, bool)  # Dirichlet face nodes are held at zero on both sides
    for ax in range(ndim):
        for side, kind in enumerate(pb.bc[ax]):
            if kind == oracle.BC_DIRICHLET:
                idx = [slice(None)] * ndim
                idx[ax] = 0 if side == 0 else shape[ax] - 1
                keep[tuple(idx)] = False
    k = keep.ravel()
    assert np.abs(M.T[np.ix_(k, k)] - MT[np.ix_(k, k)]).max() <= 1e-14 * np.abs(M).max()


@pytest.mark.parametrize("ndim", [2, 3])
def test_dot_product_variable_density(ndim):
    shape, spacing, vel, dt, kw, _, n = _case(ndim, seed=5)
    rho = _rho(shape, 3)
    rng = np.random.default_rng(11)
    s = rng.standard_normal(n)
    r = rng.standard_normal((n, len(kw["rec_pos"])))
    seis_c, _ = oracle.forward(ndim, shape, spacing, 6, vel, dt, n, wavelet=s, rho=rho, **kw)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, rho=rho, **kw)
    _, adj = A.backward(pb, r, n)
    lhs = float(np.sum(seis_c * r))
    rhs = float(np.sum(s * adj[0]))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-300)


@pytest.mark.parametrize("ndim", [2, 3])
def test_density_and_velocity_gradients_match_finite_differences(ndim):
    shape, spacing, vel, dt, kw, wav, n = _case(ndim, seed=7)
    rng = np.random.default_rng(3)
    rho = _rho(shape, 4)
    vel_true = vel * (1.0 + 0.02 * rng.standard_normal(shape))
    rho_true = rho * (1.0 + 0.05 * rng.standard_normal(shape))
    obs, _ = oracle.forward(ndim, shape, spacing, 6, vel_true, dt, n, wavelet=np.asarray(wav), rho=rho_true, **kw)
    pb = A.make_problem(ndim, shape, spacing, 6, vel, dt, rho=rho, **kw)
    J, g_c, g_rho, _ = A.adjoint_gradient_full(pb, wav, obs, n)
    assert J > 0

    def misfit(v, r):
        d, _ = oracle.forward(ndim, shape, spacing, 6, v, dt, n, wavelet=np.asarray(wav), rho=r, **kw)
        return 0.5 * float(np.sum((d - obs) ** 2))

    dv = rng.standard_normal(shape)
    eps = 1e-3
    fd = (misfit(vel + eps * dv, rho) - misfit(vel - eps * dv, rho)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g_c * dv)), rel=1e-6)
    dr = rng.standard_normal(shape)
    fd = (misfit(vel, rho + eps * dr) - misfit(vel, rho - eps * dr)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g_rho * dr)), rel=1e-6)
