"""Finite-difference weights and the stable time step, in exact arithmetic.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.3, Eq. 9-10 of the paper write the second and first derivative along an
axis as central sums of radius r = order/2 with weights v_0..v_r and w_1..w_r.
The paper does not list the weights.  They are defined here by what a central
difference of that order must do: be exact on every polynomial it can be exact
on.  The linear conditions are solved with rational arithmetic
(fractions.Fraction), so the weights are exact.

Sec. 2.2, Eq. 8 bounds the time step by 2 dx / (c_max sqrt(a)), where a is
"the sum of the finite difference coefficients" of the spatial terms.  The
reading used: a is the sum of the absolute values of all second-derivative
weights over all axes, a = ndim (|v_0| + 2 sum_j |v_j|), which is the
von Neumann bound of the scheme at the grid Nyquist wavenumber.  For unequal
spacings the same bound reads dt <= 2 / (c_max sqrt(sum_i A / h_i^2)),
A = |v_0| + 2 sum_j |v_j|, which equals Eq. 8 when all h_i are equal.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence


def _solve_exact(a: List[List[Fraction]], b: List[Fraction]) -> List[Fraction]:
    """Gauss-Jordan elimination over the rationals (small dense systems)."""
    n = len(b)
    m = [row[:] + [b[i]] for i, row in enumerate(a)]
    for col in range(n):
        piv = next(i for i in range(col, n) if m[i][col] != 0)
        m[col], m[piv] = m[piv], m[col]
        p = m[col][col]
        m[col] = [x / p for x in m[col]]
        for i in range(n):
            if i != col and m[i][col] != 0:
                f = m[i][col]
                m[i] = [x - f * y for x, y in zip(m[i], m[col])]
    return [m[i][n] for i in range(n)]


def second_derivative_weights(order: int) -> List[Fraction]:
    """[v_0, v_1, ..., v_r] of Eq. 9 for an even `order` (r = order/2).

    With unit spacing, v_0 phi(0) + sum_j v_j (phi(j) + phi(-j)) must equal
    phi''(0) for phi = x^(2m), m = 0..r (odd powers cancel by symmetry):
        m = 0:  v_0 + 2 sum_j v_j           = 0
        m = 1:  2 sum_j v_j j^2             = 2
        m > 1:  2 sum_j v_j j^(2m)          = 0
    """
    if order < 2 or order % 2:
        raise ValueError("space order must be an even integer >= 2")
    r = order // 2
    rows, rhs = [], []
    for m in range(r + 1):
        row = [Fraction(1) if m == 0 else Fraction(0)]
        row += [Fraction(2 * j ** (2 * m)) for j in range(1, r + 1)]
        rows.append(row)
        rhs.append(Fraction(2) if m == 1 else Fraction(0))
    return _solve_exact(rows, rhs)


def first_derivative_weights(order: int) -> List[Fraction]:
    """[w_1, ..., w_r] of Eq. 10, where phi'(0) ~ (1/2h) sum_j w_j (phi(j) - phi(-j)).

    Exact for phi = x^(2m+1), m = 0..r-1 (even powers cancel):
        sum_j w_j j^(2m+1) = 1 if m == 0 else 0.
    """
    if order < 2 or order % 2:
        raise ValueError("space order must be an even integer >= 2")
    r = order // 2
    rows = [[Fraction(j ** (2 * m + 1)) for j in range(1, r + 1)] for m in range(r)]
    rhs = [Fraction(1) if m == 0 else Fraction(0) for m in range(r)]
    return _solve_exact(rows, rhs)


def stencil_abs_sum(order: int) -> Fraction:
    """A = |v_0| + 2 sum_j |v_j|: one axis' share of `a` in Eq. 8."""
    v = second_derivative_weights(order)
    return abs(v[0]) + 2 * sum(abs(x) for x in v[1:])


def critical_dt(order: int, spacing: Sequence[float], c_max: float) -> float:
    """Largest stable time step of Eq. 8 (reading in the module docstring)."""
    a_axis = float(stencil_abs_sum(order))
    s = sum(a_axis / (h * h) for h in spacing)
    return 2.0 / (c_max * s ** 0.5)
