"""Kaiser-windowed sinc weights for sources and receivers (Sec. 2.4, Eq. 11-12).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A point at continuous grid coordinate s (in cells) is spread over nodes i with
weight d_i = W(i - s) sinc(i - s)  (Eq. 11), W the Kaiser window

    W(x) = I0(b sqrt(1 - (x/r)^2)) / I0(b)   for |x| <= r, else 0,

sinc(x) = sin(pi x)/(pi x).  Readings used where the paper is silent:
  - the window covers the 2r nodes floor(s)-r+1 .. floor(s)+r, i.e. every node
    with |i - s| < r (at |i - s| = r the sinc factor vanishes); an on-grid point
    reduces to the single node s with weight 1 (sinc of a nonzero integer is 0);
  - in 2D/3D the weight is the product of the per-axis 1D weights;
  - b(r): the paper prints only b = 6.31 for r = 4.  The other entries are a
    parameter table (values attributed to Hicks 2002 Table 2, unverified here).
  - coordinates are metres from the corner of the physical domain, whose first
    node is node nbl_lo along each axis: s = nbl_lo + x / h.
  - a window that sticks out of the grid only with exactly-zero weights (an
    on-grid coordinate near a face) is moved inside the grid, each nonzero
    weight staying on its node; a nonzero weight outside the grid is an error.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

KAISER_B = {1: 1.24, 2: 2.94, 3: 4.53, 4: 6.31, 5: 7.91,
            6: 9.42, 7: 10.95, 8: 12.53, 9: 14.09, 10: 14.18}


def bessel_i0(x: float) -> float:
    """Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2."""
    term = 1.0
    total = 1.0
    k = 0
    q = 0.25 * x * x
    while True:
        k += 1
        term *= q / (k * k)
        total += term
        if term < 1e-17 * total:
            return total


def kaiser_window(x: float, r: int, b: float) -> float:
    if abs(x) > r:
        return 0.0
    return bessel_i0(b * math.sqrt(1.0 - (x / r) ** 2)) / bessel_i0(b)


def sinc(x: float) -> float:
    if x == 0.0:
        return 1.0
    if x == math.floor(x):
        return 0.0
    return math.sin(math.pi * x) / (math.pi * x)


def weights_1d(s: float, r: int, b: float | None = None) -> Tuple[int, List[float]]:
    """(first node, [d_first, ..., d_first+2r-1]) for a point at cell coordinate s."""
    if b is None:
        b = KAISER_B[r]
    base = math.floor(s)
    first = base - r + 1
    return first, [kaiser_window(i - s, r, b) * sinc(i - s) for i in range(first, first + 2 * r)]


def grid_coordinate(pos_m: float, spacing: float, nbl_lo: int) -> float:
    return nbl_lo + pos_m / spacing


def fit_window(first: int, w: List[float], n: int) -> Tuple[int, List[float]]:
    """Move a window inside nodes 0..n-1 if only zero weights stick out (else ValueError)."""
    L = len(w)
    if first >= 0 and first + L <= n:
        return first, w
    if L > n:
        raise ValueError("window longer than the axis")
    new_first = min(max(first, 0), n - L)
    out = [0.0] * L
    for j, x in enumerate(w):
        node = first + j
        if new_first <= node < new_first + L:
            out[node - new_first] = x
        elif x != 0.0:
            raise ValueError("window leaves the grid with a nonzero weight")
    return new_first, out


def point_windows(positions: Sequence[Sequence[float]], ndim: int, spacing: Sequence[float],
                  nbl_lo: Sequence[int], r: int, b: float | None = None,
                  shape: Sequence[int] | None = None):
    """Per-point, per-axis (first node, weights) in (z, y, x) order.

    In 2D the y axis is a dummy of length 1: first node 0, weight [1.0].
    With `shape`, windows are fitted into the grid (see fit_window).
    Returns a list over points of [(first_z, wz), (first_y, wy), (first_x, wx)].
    """
    out = []
    for p in positions:
        if len(p) != ndim:
            raise ValueError("position has wrong dimension")
        axes = []
        for a in range(ndim):
            fw = weights_1d(grid_coordinate(p[a], spacing[a], nbl_lo[a]), r, b)
            if shape is not None:
                fw = fit_window(fw[0], fw[1], int(shape[a]))
            axes.append(fw)
        if ndim == 2:
            axes = [axes[0], (0, [1.0]), axes[1]]
        out.append(axes)
    return out
