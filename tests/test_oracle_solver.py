"""Pins of the oracle's leapfrog loop (Eq. 7) against mathematics it must obey.

- exact discrete eigenmodes of the Laplacian with Dirichlet / Neumann ghosts
  (closed-form symbol of Eq. 9), one step and many steps (closed-form
  solution of the two-level recurrence);
- the damping term of Eq. 4 (amplitude decay e^{-eta t});
- source-receiver reciprocity (symmetric discrete operator);
- mirror symmetry of a symmetric set-up;
- the homogeneous Green's functions in 2D and 3D (Sec. 2.5, V1) with
  convergence under refinement;
- second-order convergence in time (Sec. 2.5, V2) and order-p convergence in
  space (V3) with manufactured solutions;
- the variable-density operator by manufactured solutions (Sec. 2.5, V4);
- constant density through the variable-density path equals constant density;
- conservation of the discrete energy of the undamped leapfrog scheme in a
  closed Neumann box once the source has stopped.
"""
import math

import numpy as np
import pytest

import oracle
from tests import analytic


def _symbol(order, k, h):
    """Fourier symbol of Eq. 9 along one axis: (v_0 + 2 sum_j v_j cos(j k h)) / h^2."""
    v = [float(x) for x in oracle.second_derivative_weights(order)]
    return (v[0] + 2.0 * sum(v[j] * math.cos(j * k * h) for j in range(1, len(v)))) / (h * h)


def _mode(shape, spacing, kinds, m, order):
    """Separable sine (Dirichlet) or cosine (Neumann) mode fitting the grid exactly."""
    f = np.ones(shape)
    lam = 0.0
    for a, (n, h, kind, mm) in enumerate(zip(shape, spacing, kinds, m)):
        L = (n - 1) * h
        k = mm * math.pi / L
        x = np.arange(n) * h
        g = np.sin(k * x) if kind == "d" else np.cos(k * x)
        sh = [1] * len(shape)
        sh[a] = n
        f = f * g.reshape(sh)
        lam += _symbol(order, k, h)
    return f, lam


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 8), (3, 16)])
@pytest.mark.parametrize("kind", ["d", "n"])
def test_one_step_is_the_exact_symbol(ndim, order, kind):
    """p1 - p0 = kappa * symbol * mode for p0 = p_{-1} = mode (all rows incl. boundary)."""
    r = order // 2
    shape = (r + 9, r + 7, r + 11)[:ndim] if ndim == 3 else (r + 9, r + 13)
    spacing = (3.0, 4.0, 5.0)[:ndim] if ndim == 3 else (3.0, 5.0)
    m = (2, 1, 3)[:ndim] if ndim == 3 else (2, 3)
    mode, lam = _mode(shape, spacing, [kind] * ndim, m, order)
    c, dt = 700.0, 1e-3
    bc = {"d": oracle.BC_DIRICHLET, "n": oracle.BC_NEUMANN}[kind]
    bc6 = [bc] * 6 if ndim == 3 else [bc, bc, 0, 0, bc, bc]
    vel = np.full(shape, c)
    _, p1 = oracle.run_raw(ndim, shape, spacing, order, bc6, np.zeros(shape), dt, vel,
                           n_steps=1, p0=mode, pm1=mode)
    kappa = (c * dt) ** 2
    assert np.allclose(p1 - mode, kappa * lam * mode, rtol=0, atol=1e-12)


@pytest.mark.parametrize("eta", [0.0, 40.0])
def test_many_steps_follow_the_mode_recurrence(eta):
    """A Dirichlet mode obeys (1+e) a_{n+1} = (2 - kappa lam) a_n - (1-e) a_{n-1} exactly."""
    order = 8
    shape, spacing = (21, 17), (5.0, 7.0)
    mode, lam = _mode(shape, spacing, ["d", "d"], (1, 2), order)
    c, dt = 1500.0, 1e-3
    kappa = (c * dt) ** 2
    e = eta * dt
    n_steps = 300
    _, p = oracle.run_raw(2, shape, spacing, order, [1, 1, 0, 0, 1, 1], np.full(shape, eta), dt,
                          np.full(shape, c), n_steps=n_steps, p0=mode, pm1=mode)
    # closed form through the roots of (1+e) mu^2 - (2 - kappa lam) mu + (1-e) = 0
    a, b, cc = 1.0 + e, -(2.0 + kappa * lam), 1.0 - e
    disc = complex(b * b - 4 * a * cc)
    mu1 = (-b + disc ** 0.5) / (2 * a)
    mu2 = (-b - disc ** 0.5) / (2 * a)
    # a_0 = 1, a_{-1} = 1  ->  A + B = 1, A/mu1 + B/mu2 = 1
    B = (1 - 1 / mu1) / (1 / mu2 - 1 / mu1)
    A = 1 - B
    amp = (A * mu1 ** n_steps + B * mu2 ** n_steps).real
    assert np.allclose(p, amp * mode, rtol=0, atol=1e-11)
    if eta > 0:
        # Eq. 4: the damped oscillation decays like exp(-eta t), up to O((eta dt)^2)
        assert math.log(abs(mu1)) == pytest.approx(-eta * dt, rel=e * e)
        assert np.abs(p).max() < 1.5 * math.exp(-eta * n_steps * dt)


def test_reciprocity_heterogeneous_damped():
    """Dirichlet / 'none' faces make the operator symmetric: G(s->r) == G(r->s)."""
    rng = np.random.default_rng(5)
    shape, spacing, order = (40, 46), (10.0, 10.0), 8
    vel = 1500.0 + 1500.0 * rng.random(shape)
    dt = 0.4 * 10.0 / vel.max()
    nbl = [6, 6, 6, 6]
    bc = ["null_dirichlet", "none", "none", "null_dirichlet"]
    w = oracle.ricker_samples(20.0, dt, 160)
    a, b = (77.0, 123.4), (251.3, 180.0)
    s1, _ = oracle.forward(2, shape, spacing, order, vel, dt, 160, src_pos=[a], wavelet=w,
                           rec_pos=[b], nbl=nbl, bc=bc, damp_alpha=2.0, damp_degree=2)
    s2, _ = oracle.forward(2, shape, spacing, order, vel, dt, 160, src_pos=[b], wavelet=w,
                           rec_pos=[a], nbl=nbl, bc=bc, damp_alpha=2.0, damp_degree=2)
    assert np.abs(s1).max() > 1e-4
    assert np.allclose(s1, s2, rtol=0, atol=1e-12 * np.abs(s1).max())


def test_mirror_symmetry_3d():
    shape, spacing, order = (24, 21, 21), (10.0, 10.0, 10.0), 4
    dt = 0.4 * 10.0 / 2000.0
    vel = np.full(shape, 2000.0)
    vel[12:] = 2500.0
    w = oracle.ricker_samples(25.0, dt, 60)
    nbl = [0, 4, 4, 4, 4, 4]
    bc = ["null_neumann"] + ["null_dirichlet"] * 5
    rec = [(50.0, 30.0, 60.0), (50.0, 90.0, 60.0), (50.0, 60.0, 30.0), (50.0, 60.0, 90.0)]
    s, p = oracle.forward(3, shape, spacing, order, vel, dt, 60, src_pos=[(35.0, 60.0, 60.0)],
                          wavelet=w, rec_pos=rec, nbl=nbl, bc=bc, damp_alpha=1.0)
    assert np.abs(s).max() > 0
    assert np.allclose(s[:, 0], s[:, 1], rtol=0, atol=1e-14)
    assert np.allclose(s[:, 0], s[:, 2], rtol=0, atol=1e-14)
    assert np.allclose(p, p[:, ::-1, :], rtol=0, atol=1e-14)
    assert np.allclose(p, p.transpose(0, 2, 1), rtol=0, atol=1e-14)


def test_dirichlet_boundary_nodes_stay_zero():
    shape = (30, 30)
    vel = np.full(shape, 1500.0)
    dt = 0.4 * 10.0 / 1500.0
    w = oracle.ricker_samples(20.0, dt, 120)
    # a radius-2 source window at z = 1.25 cells covers the boundary row 0
    _, p = oracle.forward(2, shape, (10.0, 10.0), 8, vel, dt, 120, src_pos=[(12.5, 145.0)],
                          wavelet=w, nbl=[0, 0, 0, 0], bc=["null_dirichlet"] * 4,
                          window_radius=2)
    assert np.abs(p).max() > 0
    assert np.all(p[0] == 0) and np.all(p[-1] == 0) and np.all(p[:, 0] == 0) and np.all(p[:, -1] == 0)


def test_window_outside_grid_is_rejected():
    shape = (30, 30)
    with pytest.raises(ValueError):
        oracle.forward(2, shape, (10.0, 10.0), 8, np.full(shape, 1500.0), 1e-3, 5,
                       src_pos=[(12.5, 145.0)], wavelet=[0.0] * 5, window_radius=4)


def test_constant_density_through_variable_density_path_is_identical():
    rng = np.random.default_rng(1)
    shape = (33, 29)
    vel = 1500.0 + 500.0 * rng.random(shape)
    dt = 0.4 * 10.0 / vel.max()
    w = oracle.ricker_samples(15.0, dt, 80)
    kw = dict(src_pos=[(101.0, 133.0)], wavelet=w, rec_pos=[(40.0, 70.0)], nbl=[5, 5, 5, 5],
              bc=["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet"],
              damp_alpha=3.0)
    s1, p1 = oracle.forward(2, shape, (10.0, 10.0), 8, vel, dt, 80, **kw)
    s2, p2 = oracle.forward(2, shape, (10.0, 10.0), 8, vel, dt, 80, rho=np.full(shape, 2.3e3), **kw)
    assert np.array_equal(s1, s2) and np.array_equal(p1, p2)


def test_sponge_absorbs():
    """With the absorbing layer the late-time field is far smaller than with a bare Dirichlet box."""
    shape = (81, 81)
    vel = np.full(shape, 1500.0)
    dt = 0.4 * 10.0 / 1500.0
    n = 500
    w = oracle.ricker_samples(15.0, dt, n)
    e = {}
    for nbl, alpha in ((0, 0.0), (20, 1e-3 * 8.0)):
        shape_i = shape
        pos = [(400.0 - 10.0 * nbl, 400.0 - 10.0 * nbl)]
        _, p = oracle.forward(2, shape_i, (10.0, 10.0), 8, vel, dt, n, src_pos=pos, wavelet=w,
                              nbl=[nbl] * 4, bc=["null_dirichlet"] * 4, damp_alpha=alpha)
        e[nbl] = float(np.sum(p[20:61, 20:61] ** 2))
    assert e[20] < 1e-3 * e[0]


# ---- Green's functions (Sec. 2.5, V1) ---------------------------------------

def _green_case_2d(h, f=20.0, c=1500.0, t_end=0.25):
    L = 500.0
    n = int(round(L / h)) + 1
    shape = (n, n)
    dt = 0.4 * h / c
    steps = int(round(t_end / dt))
    t0 = 1.5 / f
    w = oracle.ricker_samples(f, dt, steps, t0=t0)
    src = (250.0, 250.0)
    rec = (250.0 + 60.0, 250.0 + 80.0)  # 100 m away
    s, _ = oracle.forward(2, shape, (h, h), 8, np.full(shape, c), dt, steps, src_pos=[src],
                          wavelet=w, rec_pos=[rec], nbl=[0, 0, 0, 0], bc=["null_dirichlet"] * 4)
    t = (np.arange(steps) + 1) * dt
    ref = np.array([analytic.green_2d(100.0, tt, c, f, t0) for tt in t])
    return np.linalg.norm(s[:, 0] - ref) / np.linalg.norm(ref)


def test_green_2d_and_refinement():
    e1 = _green_case_2d(5.0)
    e2 = _green_case_2d(2.5)
    assert e1 < 3e-2
    assert e2 < 0.5 * e1


def test_green_3d():
    h, c, f = 10.0, 1500.0, 10.0
    n = 81
    shape = (n, n, n)
    dt = 0.4 * h / c
    t_end = 0.42
    steps = int(round(t_end / dt))
    t0 = 1.5 / f
    w = oracle.ricker_samples(f, dt, steps, t0=t0)
    src = (400.0, 400.0, 400.0)
    rec = (400.0 + 60.0, 400.0 - 48.0, 400.0 + 64.0)  # 100 m away
    s, _ = oracle.forward(3, shape, (h, h, h), 8, np.full(shape, c), dt, steps, src_pos=[src],
                          wavelet=w, rec_pos=[rec], nbl=[0] * 6, bc=["null_dirichlet"] * 6)
    t = (np.arange(steps) + 1) * dt
    ref = np.array([analytic.green_3d(100.0, tt, c, f, t0) for tt in t])
    assert np.linalg.norm(s[:, 0] - ref) / np.linalg.norm(ref) < 3e-2


# ---- convergence (Sec. 2.5, V2-V4) -------------------------------------------

def _mms_error(order, h, dt, t_end, density, c=2000.0, L=440.0):
    n = int(round(L / h)) + 1
    steps = int(round(t_end / dt))
    rho, F, T, uN = analytic.mms_2d(L, c, n, n, h, dt, steps, density)
    _, p = oracle.forward(2, (n, n), (h, h), order, np.full((n, n), c), dt, steps, nbl=[0] * 4,
                          bc=["null_dirichlet"] * 4, rho=rho, force_fields=F, force_sigs=T)
    # normalise by the spatial shape (|T(t)| <= 1), not by u*(t_N), which can vanish
    shape_norm = np.linalg.norm(analytic.mms_2d(L, c, n, n, h, dt, 0, None)[1][0]) * c * c
    return np.linalg.norm(p - uN) / shape_norm


def test_time_convergence_second_order():
    """V2: space error negligible (order 16, fine grid); halving dt quarters the error."""
    errs = [_mms_error(16, 11.0, dt, 0.1, None) for dt in (8e-4, 4e-4, 2e-4)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < r < 2.1 for r in rates), (errs, rates)


@pytest.mark.parametrize("order", [2, 4])
def test_space_convergence_order(order):
    """V3: time error negligible (dt = 5 us); halving h divides the error by about 2^order."""
    errs = [_mms_error(order, h, 5e-6, 0.02, None) for h in (44.0, 22.0)]
    rate = math.log2(errs[0] / errs[1])
    assert order - 0.4 < rate < order + 0.4, (errs, rate)


def test_variable_density_mms_interior_order():
    """Strong density contrast whose ln is even at the walls: about 4th-order convergence."""
    errs = [_mms_error(4, h, 5e-6, 0.02, "cos") for h in (44.0, 22.0, 11.0)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.5 < r < 4.4 for r in rates), (errs, rates)
    # the advective term matters: solving without it misses by far more
    errs_wrong = _mms_error(4, 11.0, 5e-6, 0.02, "cos_ignored")
    assert errs_wrong > 1000 * errs[2]


def test_variable_density_mms_paper_setup():
    """V4 as in the paper (Eq. 14-15, c = 2 km/s, 440 m box): error falls under refinement."""
    errs = [_mms_error(8, h, 5e-5, 0.05, "paper") for h in (40.0, 20.0, 10.0)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-6


# Textbook central second-derivative weights v_0 .. v_R (orders 4 and 8),
# written out here independently of the oracle's rational solve.
_V_TEXTBOOK = {4: [-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0],
               8: [-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0]}


def _neumann_laplacian(p, spacing, order):
    """Eq. 9 with even ghosts (p[-j] = p[j] about every face node)."""
    v = _V_TEXTBOOK[order]
    R = len(v) - 1
    out = np.zeros_like(p)
    for a, h in enumerate(spacing):
        q = np.pad(p, [(R, R) if b == a else (0, 0) for b in range(p.ndim)], mode="reflect")
        n = p.shape[a]
        acc = v[0] * p
        for j in range(1, R + 1):
            acc = acc + v[j] * (np.take(q, np.arange(R + j, R + j + n), axis=a) +
                                np.take(q, np.arange(R - j, R - j + n), axis=a))
        out += acc / (h * h)
    return out


def _face_weights(shape):
    """Diagonal W with 1/2 per axis on face nodes: W L is symmetric for even ghosts."""
    w = np.ones(shape)
    for a, n in enumerate(shape):
        g = np.ones(n)
        g[0] = g[-1] = 0.5
        sh = [1] * len(shape)
        sh[a] = n
        w = w * g.reshape(sh)
    return w


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 8)])
def test_energy_conserved_in_closed_neumann_box(ndim, order):
    """With no absorbing layer (eta = 0, Eq. 4) and Neumann ghosts on every face,
    the leapfrog recurrence of Eq. 7, p+ = 2p - p- + kappa L p, conserves
    E = sum W/kappa (p+ - p)^2 - sum W p+ (L p) (W: face weights that make W L
    symmetric), so E taken at two times after the source has stopped agrees to
    round-off; a wrong ghost sign, weight or index in the oracle breaks it."""
    rng = np.random.default_rng(11 + ndim + order)
    if ndim == 2:
        shape, spacing = (34, 41), (8.0, 10.0)
        src = [(0.43 * 33 * 8.0, 0.57 * 40 * 10.0)]
    else:
        shape, spacing = (17, 19, 21), (9.0, 10.0, 8.0)
        src = [(0.45 * 16 * 9.0, 0.5 * 18 * 10.0, 0.55 * 20 * 8.0)]
    vel = 1500.0 + 1000.0 * rng.random(shape)
    dt = 0.3 * min(spacing) / vel.max()
    w = np.zeros(400)
    w[:24] = oracle.ricker_samples(40.0, dt, 24, t0=12 * dt)  # a source that stops after 24 steps
    kw = dict(src_pos=src, wavelet=w, nbl=[0] * (2 * ndim), bc=["null_neumann"] * (2 * ndim),
              window_radius=3)
    kappa = (vel * dt) ** 2
    W = _face_weights(shape)

    def energy(n):
        _, p1, p0 = oracle.forward(ndim, shape, spacing, order, vel, dt, n, want_prev=True, **kw)
        return float(np.sum(W / kappa * (p1 - p0) ** 2) - np.sum(W * p1 * _neumann_laplacian(p0, spacing, order)))

    e1, e2, e3 = energy(60), energy(170), energy(300)
    assert e1 > 0
    assert abs(e2 - e1) <= 1e-9 * e1 and abs(e3 - e1) <= 1e-9 * e1



# ---- sources and forcing inside a damped region (Eq. 4, 7, 11) ---------------
#
# With a uniform eta and uniform kappa, every Dirichlet sine (Neumann cosine)
# mode is an eigenvector of the Eq. 9 operator, so projecting Eq. 7 with a
# source or forcing term onto a mode leaves the scalar recurrence
#   (1 + e) a[n+1] = (2 - kappa lam) a[n] - (1 - e) a[n-1] + kappa g[n],
# e = eta dt, g[n] the term's projection onto the mode.  The recurrence is
# solved here by a scalar loop per mode; the oracle must give the same field.
# Dropping the 1/(1 + e) from the oracle's source or forcing term, or applying
# it to the forcing but not to the point source, fails these tests.


def _forced_amplitudes(kappa, lam, e, g):
    """a[1..N] of the forced, damped two-level recurrence from a[0] = a[-1] = 0;
    lam and g[n] may be arrays over modes (g has the step as its first axis)."""
    lam = np.asarray(lam, dtype=np.float64)
    a_prev = np.zeros_like(lam)
    a = np.zeros_like(lam)
    out = []
    for gn in g:
        a_next = ((2.0 - kappa * lam) * a - (1.0 - e) * a_prev + kappa * gn) / (1.0 + e)
        a_prev, a = a, a_next
        out.append(a)
    return out


@pytest.mark.parametrize("ndim,kind,order", [(2, "d", 8), (2, "n", 4), (3, "d", 8), (3, "n", 16)])
def test_forced_mode_under_uniform_damping(ndim, kind, order):
    """Forcing F(x) T(t_n) with F a mode and eta > 0 everywhere: p[n] = a[n] F."""
    r = order // 2
    shape = (r + 14, r + 11, r + 16)[:ndim] if ndim == 3 else (r + 17, r + 21)
    spacing = (6.0, 7.0, 5.0)[:ndim] if ndim == 3 else (6.0, 5.0)
    m = (2, 1, 3)[:ndim] if ndim == 3 else (1, 2)
    mode, lam = _mode(shape, spacing, [kind] * ndim, m, order)
    lam = -lam  # _mode returns the symbol (negative); the recurrence uses L mode = -lam mode
    c, dt, eta = 1200.0, 1e-3, 150.0  # e = 0.15
    kappa, e = (c * dt) ** 2, eta * dt
    n_steps = 90
    T = np.random.default_rng(7 + ndim).standard_normal(n_steps)
    bc = {"d": oracle.BC_DIRICHLET, "n": oracle.BC_NEUMANN}[kind]
    bc6 = [bc] * 6 if ndim == 3 else [bc, bc, 0, 0, bc, bc]
    _, p, p_prev = oracle.run_raw(ndim, shape, spacing, order, bc6, np.full(shape, eta), dt, np.full(shape, c),
                                  n_steps=n_steps, force_fields=mode[None], force_sigs=T[None], want_prev=True)
    a = _forced_amplitudes(kappa, lam, e, T)
    scale = max(abs(a[-1]), abs(a[-2]))
    assert scale > 1e-3
    assert np.allclose(p, a[-1] * mode, rtol=0, atol=1e-11 * scale)
    assert np.allclose(p_prev, a[-2] * mode, rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("on_grid", [True, False])
def test_point_source_under_uniform_damping_by_sine_modes(on_grid):
    """A point source (Eq. 11) in a Dirichlet box with eta > 0 everywhere: the
    oracle's field equals the sum over the box's sine modes of the forced,
    damped scalar recurrence driven by the source pattern's projection."""
    order = 8
    shape, spacing = (23, 27), (8.0, 6.0)
    nz, nx = shape
    c, dt, eta = 1500.0, 1.2e-3, 110.0  # e = 0.132
    kappa, e = (c * dt) ** 2, eta * dt
    n_steps = 70
    # on-grid: one node of weight 1; off-grid: the product of the two 1D windows
    pos = (9.0 * 8.0, 14.0 * 6.0) if on_grid else (9.37 * 8.0, 13.61 * 6.0)
    wins = oracle.point_windows([pos], 2, spacing, [0, 0], 3, shape=shape)
    (fz, wz), _, (fx, wx) = wins[0]
    pattern = np.zeros(shape)
    pattern[fz:fz + len(wz), fx:fx + len(wx)] = np.outer(wz, wx) / (spacing[0] * spacing[1])
    assert np.count_nonzero(pattern) == (1 if on_grid else 36)
    assert not pattern[0].any() and not pattern[-1].any() and not pattern[:, 0].any() and not pattern[:, -1].any()
    S = oracle.ricker_samples(60.0, dt, n_steps, t0=0.02)
    _, p = oracle.run_raw(2, shape, spacing, order, [1, 1, 0, 0, 1, 1], np.full(shape, eta), dt,
                          np.full(shape, c), src_windows=wins, src_sig=S, n_steps=n_steps)
    # sine basis of the interior nodes: phi_m(i) = sin(pi m i / (n - 1)), m = 1 .. n-2,
    # orthogonal with sum_i phi_m phi_m' = (n - 1) / 2 delta_mm'
    def basis(n):
        i = np.arange(n)[:, None]
        mm = np.arange(1, n - 1)[None, :]
        return np.sin(np.pi * mm * i / (n - 1)), mm[0]

    Pz, mz = basis(nz)
    Px, mx = basis(nx)
    coef = (2.0 / (nz - 1)) * (2.0 / (nx - 1)) * (Pz.T @ pattern @ Px)  # [mode_z, mode_x]
    assert np.allclose(Pz @ coef @ Px.T, pattern, rtol=0, atol=1e-12 * np.abs(pattern).max())
    lam = -(np.array([_symbol(order, k * np.pi / ((nz - 1) * spacing[0]), spacing[0]) for k in mz])[:, None] +
            np.array([_symbol(order, k * np.pi / ((nx - 1) * spacing[1]), spacing[1]) for k in mx])[None, :])
    a = _forced_amplitudes(kappa, lam, e, [s * coef for s in S])[-1]
    expect = Pz @ a @ Px.T
    assert np.abs(expect).max() > 1e-6
    assert np.allclose(p, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


def test_first_step_of_sources_in_the_absorbing_layer():
    """One step from rest: p[1] = kappa/(1 + eta dt) S(t_0) d_k / prod(h) at every
    window node (Eq. 7, Eq. 11) with the layer's eta (Eq. 4) at that node, and
    zero elsewhere; two sources deep in the layer, one in the physical box."""
    shape, spacing = (30, 34), (10.0, 8.0)
    nbl = [0, 8, 7, 8]
    rng = np.random.default_rng(3)
    vel = 1600.0 + 900.0 * rng.random(shape)
    dt = 0.35 * 8.0 / vel.max()
    alpha, deg = 9.0, 3
    # cell coordinates (z, x): (10.3, 3.2) in the x- layer, (25.4, 15.6) in the
    # z+ layer, (12.2, 16.7) in the physical box (x node 7 is its first column)
    src = [(10.3 * 10.0, (3.2 - 7) * 8.0), (25.4 * 10.0, (15.6 - 7) * 8.0), (12.2 * 10.0, (16.7 - 7) * 8.0)]
    S0 = 0.73
    _, p = oracle.forward(2, shape, spacing, 8, vel, dt, 1, src_pos=src, wavelet=[S0], nbl=nbl,
                          bc=["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet"],
                          damp_alpha=alpha, damp_degree=deg, window_radius=3)
    eta = oracle.eta_field(shape, nbl, alpha, deg)
    expect = np.zeros(shape)
    for axes in oracle.point_windows(src, 2, spacing, [nbl[0], nbl[2]], 3, shape=shape):
        (fz, wz), _, (fx, wx) = axes
        expect[fz:fz + len(wz), fx:fx + len(wx)] += np.outer(wz, wx) * S0 / (spacing[0] * spacing[1])
    kap = (vel * dt) ** 2
    expect *= kap / (1.0 + eta * dt)
    e_src = (eta * dt)[expect != 0]
    assert e_src.max() > 0.05  # some source nodes are strongly damped
    assert np.allclose(p, expect, rtol=0, atol=1e-14 * np.abs(expect).max())
