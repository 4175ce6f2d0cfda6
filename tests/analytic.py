"""Closed-form solutions used to pin the oracle (not imported by product code).

- Homogeneous Green's functions of p_tt - c^2 Lap p = c^2 S(t) delta(x), the
  continuous problem the discrete source of Eq. 11 approximates (Sec. 2.5,
  Eq. 13 states the 2D case in the frequency domain; the time-domain forms
  below are the textbook equivalents and avoid the garbled prefactor):
    2D: p(r, t) = (1/2pi) int_0^{acosh(ct/r)} S(t - (r/c) cosh th) d th
    3D: p(r, t) = S(t - r/c) / (4 pi r)
- Manufactured solutions for Eq. 5 (Sec. 2.5, Eq. 14-15) with a distributed
  forcing split into separable terms F_m(x) T_m(t).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def ricker(f, t, t0):
    a = (math.pi * f * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def green_2d(r, t, c, f, t0):
    if c * t <= r:
        return 0.0
    top = math.acosh(c * t / r)
    val, _ = integrate.quad(lambda th: ricker(f, t - (r / c) * math.cosh(th), t0), 0.0, top,
                            limit=400, epsabs=1e-12, epsrel=1e-10)
    return val / (2.0 * math.pi)


def green_3d(r, t, c, f, t0):
    return ricker(f, t - r / c, t0) / (4.0 * math.pi * r)


def mms_2d(L, c, nz, nx, h, dt, n_steps, density):
    """Forcing terms and exact final field for u* = sin(pi x/L) sin(pi z/L) T(t).

    T(t) = sin(20 pi t) sin(20 pi (t + dt)) (Eq. 15 as printed), which vanishes
    at the two initial levels t_{-1} = -dt and t_0 = 0 of the leapfrog scheme.
    density: None (constant), "paper" (Eq. 14) or "cos" ((2+cos)(2+cos), whose
    ln is even about both walls); "cos_ignored" builds the "cos" forcing but
    returns rho = None (a deliberately wrong model, to show the term matters).
    Returns rho, force_fields [2, nz, nx], force_sigs [2, n_steps], u*(t_N).
    """
    z = np.arange(nz)[:, None] * h
    x = np.arange(nx)[None, :] * h
    k = math.pi / L
    X, Z = np.sin(k * x), np.sin(k * z)
    u = Z * X
    lap_u = -2.0 * k * k * u
    ux = Z * k * np.cos(k * x)
    uz = k * np.cos(k * z) * X
    if density is None:
        rho = None
        adv = np.zeros_like(u)
    elif density == "paper":
        rho = (1000.0 + np.sin(k * x)) * (1000.0 + np.sin(k * z))
        gx = k * np.cos(k * x) / (1000.0 + np.sin(k * x))
        gz = k * np.cos(k * z) / (1000.0 + np.sin(k * z))
        adv = gx * ux + gz * uz
    elif density in ("cos", "cos_ignored"):
        rho = (2.0 + np.cos(k * x)) * (2.0 + np.cos(k * z))
        gx = -k * np.sin(k * x) / (2.0 + np.cos(k * x))
        gz = -k * np.sin(k * z) / (2.0 + np.cos(k * z))
        adv = gx * ux + gz * uz
    else:
        raise ValueError(density)
    a = 20.0 * math.pi
    t = np.arange(n_steps) * dt
    T = np.sin(a * t) * np.sin(a * (t + dt))
    Tpp = 2.0 * a * a * np.cos(a * (2.0 * t + dt))
    F1 = u / (c * c)
    F2 = adv - lap_u
    tN = n_steps * dt
    uN = u * math.sin(a * tN) * math.sin(a * (tN + dt))
    if density == "cos_ignored":  # forcing of the variable-density problem, solver told rho = const
        rho = None
    rho_full = None if rho is None else np.broadcast_to(rho, (nz, nx)).copy()
    return rho_full, np.stack([F1, F2]), np.stack([Tpp, T]), uN
