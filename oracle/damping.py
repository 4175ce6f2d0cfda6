"""Absorbing-layer damping profile (Sec. 2.1, Eq. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

eta(x) = alpha d(x)^p inside the absorbing layer and 0 in the physical domain,
d(x) the shortest distance from x to the physical domain.  Reading used: d is
measured in grid cells (in metres the paper's own example, alpha = 0.001,
p = 3, 700 m layer, gives eta dt of several hundred), and the shortest distance
to the box of physical nodes is the Euclidean one, so in an edge or corner
region d^2 is the sum of the per-axis squared distances.

The physical nodes along an axis with n nodes are nbl_lo .. n-1-nbl_hi.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def distance_to_interior(shape: Sequence[int], nbl: Sequence[int]) -> np.ndarray:
    """d(x) in cells for every node; nbl lists (lo, hi) per axis in (z, [y,] x) order."""
    ndim = len(shape)
    d2 = np.zeros(tuple(shape), dtype=np.float64)
    for a in range(ndim):
        n = shape[a]
        lo, hi = nbl[2 * a], nbl[2 * a + 1]
        i = np.arange(n)
        da = np.zeros(n, dtype=np.float64)
        da[i < lo] = (lo - i[i < lo])
        last = n - 1 - hi
        da[i > last] = (i[i > last] - last)
        sh = [1] * ndim
        sh[a] = n
        d2 = d2 + (da ** 2).reshape(sh)
    return np.sqrt(d2)


def eta_field(shape: Sequence[int], nbl: Sequence[int], alpha: float, degree: int) -> np.ndarray:
    d = distance_to_interior(shape, nbl)
    return alpha * d ** degree
