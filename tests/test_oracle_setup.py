"""Pins of the oracle's setup routines (FD weights, dt, Kaiser-sinc, Ricker, damping).

Each check compares the oracle against something independent of it: textbook
values, a closed form derived differently, a library routine, the paper's
printed numbers, or brute force.
"""
import math
import os
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.signal
import scipy.special

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---- FD weights (Eq. 9-10) -------------------------------------------------

def test_fd_weights_textbook_values():
    for row in _golden_lines("fd_weights.txt"):
        kind, order, vals = row[0], int(row[1]), [Fraction(v) for v in row[2:]]
        if kind == "d2":
            assert oracle.second_derivative_weights(order) == vals
        else:
            # Eq. 10 carries 1/(2h): w_j = 2 * (textbook 1/h weight)
            assert oracle.first_derivative_weights(order) == [2 * v for v in vals[1:]]


@pytest.mark.parametrize("order", range(2, 21, 2))
def test_fd_weights_closed_form(order):
    """Closed form of the central weights (Fornberg 1988 / Lagrange derivation)."""
    M = order // 2
    v = oracle.second_derivative_weights(order)
    w = oracle.first_derivative_weights(order)
    for j in range(1, M + 1):
        vj = Fraction(2 * (-1) ** (j + 1) * factorial(M) ** 2,
                      j * j * factorial(M - j) * factorial(M + j))
        wj = Fraction(2 * (-1) ** (j + 1) * factorial(M) ** 2,
                      j * factorial(M - j) * factorial(M + j))
        assert v[j] == vj
        assert w[j - 1] == wj
    assert v[0] == -2 * sum(v[1:])


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_fd_order_of_accuracy(order):
    """Exact on polynomials up to degree order+1 about an off-grid centre, not beyond."""
    v = oracle.second_derivative_weights(order)
    w = oracle.first_derivative_weights(order)
    r = order // 2
    c, h = Fraction(2, 7), Fraction(1, 3)
    for k in range(order + 3):
        f = lambda x: x ** k  # noqa: E731
        d2 = (v[0] * f(c) + sum(v[j] * (f(c + j * h) + f(c - j * h)) for j in range(1, r + 1))) / h ** 2
        d1 = sum(w[j - 1] * (f(c + j * h) - f(c - j * h)) for j in range(1, r + 1)) / (2 * h)
        exact2 = k * (k - 1) * c ** (k - 2) if k >= 2 else Fraction(0)
        exact1 = k * c ** (k - 1) if k >= 1 else Fraction(0)
        if k <= order + 1:
            assert d2 == exact2
        if k <= order:
            assert d1 == exact1
    # degree order+2 is not reproduced: the scheme is of order `order`, not higher
    k = order + 2
    f = lambda x: x ** k  # noqa: E731
    d2 = (v[0] * f(c) + sum(v[j] * (f(c + j * h) + f(c - j * h)) for j in range(1, r + 1))) / h ** 2
    assert d2 != k * (k - 1) * c ** (k - 2)


# ---- stable time step (Eq. 8) ----------------------------------------------

def test_cfl_reproduces_paper_step_counts():
    """One c_max per benchmark must give all three printed step counts (ceil(tf/dt))."""
    rows = _golden_lines("paper_step_counts.txt")
    for ndim in (2, 3):
        lo, hi = 0.0, float("inf")
        for r in rows:
            if int(r[0]) != ndim:
                continue
            h, tf, order, steps = float(r[1]), float(r[2]), int(r[3]), int(r[4])
            # ceil(tf/dt) == steps  <=>  steps-1 < tf/dt <= steps; tf/dt is linear in c_max
            per_c = tf / oracle.critical_dt(order, [h] * ndim, 1.0)
            lo = max(lo, (steps - 1) / per_c)
            hi = min(hi, steps / per_c)
        assert lo < hi, "no single c_max reproduces the printed counts"
        # the implied maximum velocities are the benchmark models' (about 4.7 and 6.0 km/s)
        assert {2: 4600 < lo < 4800, 3: 5900 < lo < 6100}[ndim]


def test_cfl_is_the_von_neumann_limit():
    """At dt slightly above the bound a Nyquist checkerboard grows, slightly below it does not."""
    order, h, c = 8, 10.0, 1500.0
    n = 17
    dtc = oracle.critical_dt(order, [h, h], c)
    zz, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    chk = (-1.0) ** (zz + xx)
    vel = np.full((n, n), c)
    eta = np.zeros((n, n))
    growth = {}
    for f in (0.98, 1.02):
        _, p = oracle.run_raw(2, (n, n), (h, h), order, [2, 2, 0, 0, 2, 2], eta, f * dtc, vel,
                              n_steps=400, p0=chk, pm1=chk)
        growth[f] = np.abs(p).max()
    assert growth[0.98] < 10.0
    assert growth[1.02] > 1e3


# ---- Kaiser-windowed sinc (Eq. 11-12) --------------------------------------

def test_bessel_i0_matches_library():
    for x in np.linspace(0.0, 30.0, 61):
        assert oracle.bessel_i0(float(x)) == pytest.approx(float(scipy.special.i0(x)), rel=1e-14)


def test_kaiser_b_from_paper():
    for r, b in _golden_lines("kaiser.txt"):
        assert oracle.KAISER_B[int(r)] == float(b)


def test_kaiser_window_shape():
    r, b = 4, 6.31
    assert oracle.kaiser_window(0.0, r, b) == 1.0
    assert oracle.kaiser_window(r, r, b) == pytest.approx(1.0 / scipy.special.i0(b), rel=1e-14)
    assert oracle.kaiser_window(r + 0.01, r, b) == 0.0
    for x in (0.3, 1.7, 3.2):
        assert oracle.kaiser_window(x, r, b) == oracle.kaiser_window(-x, r, b)
    # scipy's Kaiser window (beta = b) sampled at the same abscissae
    M = 9
    ref = scipy.signal.windows.kaiser(M, b, sym=True)
    xs = np.linspace(-r, r, M)
    got = [oracle.kaiser_window(float(x), r, b) for x in xs]
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)



def test_on_grid_point_is_a_kronecker_delta():
    for r in range(1, 11):
        first, w = oracle.weights_1d(7.0, r)
        assert first == 7 - r + 1 and len(w) == 2 * r
        assert w[r - 1] == 1.0
        assert all(x == 0.0 for i, x in enumerate(w) if i != r - 1)


def test_off_grid_weights_symmetry_and_interpolation():
    r = 4
    for alpha in (0.1, 0.25, 0.5):
        f1, w1 = oracle.weights_1d(10.0 + alpha, r)
        f2, w2 = oracle.weights_1d(10.0 + (1.0 - alpha), r)
        # mirror image about the midpoint between nodes 10 and 11
        assert np.allclose(w1, w2[::-1], rtol=0, atol=1e-15)
        # band-limited delta: gain close to 1 and accurate interpolation of
        # wavenumbers below pi/2 (the design band of the b table)
        s = 10.0 + alpha
        assert abs(sum(w1) - 1.0) < 2e-3
        for k in (0.2 * math.pi, 0.4 * math.pi):
            nodes = np.arange(f1, f1 + 2 * r)
            est = float(np.dot(w1, np.cos(k * (nodes - s))))
            assert abs(est - 1.0) < 2e-2


def test_point_windows_2d_layout():
    wins = oracle.point_windows([(20.0, 35.0)], 2, [10.0, 10.0], [3, 5], 2)
    (fz, wz), (fy, wy), (fx, wx) = wins[0]
    assert (fy, wy) == (0, [1.0])
    assert fz == 5 - 2 + 1 and wz[1] == 1.0  # on-grid in z: node 3 + 2 = 5
    assert fx == 8 - 2 + 1 and len(wx) == 4  # x: 5 + 3.5 = 8.5


# ---- Ricker wavelet ---------------------------------------------------------

def test_ricker_is_second_derivative_of_gaussian():
    f, t0 = 12.0, 0.1
    a = (math.pi * f) ** 2
    h = 1e-5
    for t in np.linspace(0.0, 0.2, 21):
        g = lambda s: math.exp(-a * (s - t0) ** 2)  # noqa: E731
        d2 = (g(t + h) - 2 * g(t) + g(t - h)) / h ** 2
        assert oracle.ricker(f, float(t), t0) == pytest.approx(-d2 / (2 * a), abs=2e-5)


def test_ricker_spectrum_peaks_at_f():
    f, dt, nt = 15.0, 1e-4, 1 << 16
    s = np.array(oracle.ricker_samples(f, dt, nt, t0=0.2))
    spec = np.abs(np.fft.rfft(s))
    freqs = np.fft.rfftfreq(nt, dt)
    assert abs(freqs[np.argmax(spec)] - f) < 0.2


# ---- damping profile (Eq. 4) -------------------------------------------------

def test_damping_distance_brute_force():
    shape, nbl = (9, 7, 8), [2, 3, 0, 2, 1, 2]
    d = oracle.distance_to_interior(shape, nbl)
    inner = [(z, y, x) for z in range(shape[0]) for y in range(shape[1]) for x in range(shape[2])
             if nbl[0] <= z < shape[0] - nbl[1] and nbl[2] <= y < shape[1] - nbl[3]
             and nbl[4] <= x < shape[2] - nbl[5]]
    inner = np.array(inner, dtype=float)
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                ref = np.sqrt(((inner - [z, y, x]) ** 2).sum(1)).min()
                assert d[z, y, x] == pytest.approx(ref, abs=1e-12)
    eta = oracle.eta_field(shape, nbl, 0.5, 3)
    assert np.allclose(eta, 0.5 * d ** 3)
    assert eta[nbl[0]:shape[0] - nbl[1], nbl[2]:shape[1] - nbl[3], nbl[4]:shape[2] - nbl[5]].max() == 0


def test_window_fitting_keeps_nonzero_weights_on_their_nodes():
    # on-grid in z at node 2 with r = 4: nodes -1..6, only node 2 is nonzero
    f, w = oracle.weights_1d(2.0, 4)
    assert f == -1
    f2, w2 = oracle.source.fit_window(f, w, 50)
    assert f2 == 0 and w2[2] == 1.0 and sum(abs(x) for x in w2) == 1.0
    # high face: node 47 of 50, nodes 44..51
    f, w = oracle.weights_1d(47.0, 4)
    f2, w2 = oracle.source.fit_window(f, w, 50)
    assert f2 == 42 and w2[47 - 42] == 1.0
    # off-grid near the face: a nonzero weight would leave the grid
    f, w = oracle.weights_1d(2.5, 4)
    with pytest.raises(ValueError):
        oracle.source.fit_window(f, w, 50)
