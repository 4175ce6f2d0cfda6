"""Ricker wavelet (Sec. 2.4: the default time signal for a user-chosen peak frequency).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names the Ricker wavelet and its peak frequency but not its formula
or delay.  Reading used: S(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
tau = t - t0, unit peak amplitude, delay t0 (default 1/f).  Samples are taken
at t_n = n dt.
"""
from __future__ import annotations

import math
from typing import List


def ricker(f_peak: float, t: float, t0: float | None = None) -> float:
    if t0 is None:
        t0 = 1.0 / f_peak
    a = (math.pi * f_peak * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def ricker_samples(f_peak: float, dt: float, nt: int, t0: float | None = None) -> List[float]:
    return [ricker(f_peak, n * dt, t0) for n in range(nt)]
