"""FP64 adjoint-state gradient of the seismogram misfit.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Extension beyond the paper (the paper names FWI as a use, Sec. 1 and 6, but
prints no adjoint): the exact discrete adjoint of the forward recurrence that
oracle.c steps through, written out in numpy.

Forward, n = 0 .. N-1 (Sec. 2.2-2.4, Eq. 7, 9, 11, 12):
    p[n+1] = Z( a (2 p[n] + kappa L p[n] - (1 - e) p[n-1]) + a kappa s[n] )
    d[n]   = R p[n+1]
  a = 1/(1+e), e = eta dt, kappa = c^2 dt^2; L the Eq. 9 Laplacian on node
  values whose ghosts follow the face conditions (Dirichlet odd mirror,
  Neumann even mirror, none zero); Z zeroes Dirichlet face nodes; s[n] the
  source window weights / prod(h) times S(t_n); R the receiver weights.
Misfit J = 1/2 sum_n |d[n] - d_obs[n]|^2, residual r[n] = d[n] - d_obs[n].

Adjoint: with lambda[k] = dJ/dp[k] restricted by Z and psi = kappa a lambda,
    psi[k] = Z( a (2 psi[k+1] + kappa L^T psi[k+1] - (1 - e) psi[k+2])
                + kappa a R^T r[k-1] ),   k = N .. 1,  psi[N+1] = psi[N+2] = 0,
the forward update with L^T for L and the residuals injected through the
receiver weights.  L^T equals L with the same ghost mirrors except along a
Neumann face, where the even mirror makes L non-symmetric: the face node's
own row has both halves of its stencil on the interior side (2 v_j), while
node j reaches the face node once.  Hence, per Neumann face and axis with
spacing h, L^T f = L f + v_k / h^2 f_face at the nodes k = 1..R from the face
and L^T f = L f - sum_j v_j / h^2 f_j at the face node.  (Along a Dirichlet
face the only asymmetric entries involve the face node, which Z holds at 0.)
Gradient: dJ/dkappa = sum_{n=0}^{N-1} psi[n+1] (L p[n] + s[n]) / kappa and
dJ/dc = 2 c dt^2 dJ/dkappa.

Variable density (Eq. 5 with Eq. 10): the forward operator is
    L_rho p = L p - sum_a G_a D_a p,   G_a = D_a^even ln(rho),
D_a the first derivative of Eq. 10 along axis a on node values whose ghosts
follow the face conditions, D_a^even the same with even ghosts on every face
(how the solver extends ln rho).  Its transpose is
    L_rho^T q = L^T q - sum_a D_a^T (G_a q),
where D_a^T is the literal transpose of "fill the ghosts, then take the
centred difference": scatter each node's difference weights onto the
extended array, then fold every ghost back onto the node it mirrors, with
the mirror's sign.  The adjoint sweep uses L_rho^T for L^T; dJ/dkappa uses
L_rho p[n]; and with dJ/dG_a = - sum_n psi[n+1] D_a p[n],
    dJ/d ln(rho) = sum_a (D_a^even)^T dJ/dG_a,   dJ/drho = dJ/d ln(rho) / rho.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from .damping import eta_field
from .fd import first_derivative_weights, second_derivative_weights
from .solver import BC_DIRICHLET, BC_NEUMANN, BC_NONE, _bc_codes
from .source import KAISER_B, point_windows


@dataclass
class Problem:
    ndim: int
    shape: tuple
    spacing: tuple
    R: int
    v: np.ndarray        # second-derivative weights v_0 .. v_R
    bc: list             # per axis of the array (low, high)
    vel: np.ndarray
    kappa: np.ndarray
    a: np.ndarray        # 1 / (1 + eta dt)
    e: np.ndarray        # eta dt
    dt: float
    src: list            # per source: (first per axis, weights per axis)
    rec: list
    cell: float          # product of the spacings
    w: np.ndarray = None        # first-derivative weights 0, w_1 .. w_R (Eq. 10)
    rho: np.ndarray = None      # density, or None for constant density
    G: list = None              # D_a^even ln(rho) per axis


def make_problem(ndim, shape, spacing, order, vel, dt, src_pos=(), rec_pos=(), nbl=None, bc=None,
                 damp_alpha=0.0, damp_degree=3, window_radius=4, rho=None) -> Problem:
    """Same set-up as oracle.forward."""
    shape = tuple(int(s) for s in shape)
    nbl = nbl if nbl is not None else [0] * (2 * ndim)
    bc = _bc_codes(bc if bc is not None else [BC_DIRICHLET] * (2 * ndim))
    eta = eta_field(shape, nbl, damp_alpha, damp_degree)
    e = eta * dt
    vel = np.asarray(vel, dtype=np.float64).reshape(shape)
    nbl_lo = [nbl[2 * k] for k in range(ndim)]
    b = KAISER_B[window_radius]
    sw = point_windows(src_pos, ndim, spacing, nbl_lo, window_radius, b, shape)
    rw = point_windows(rec_pos, ndim, spacing, nbl_lo, window_radius, b, shape)
    drop_y = (lambda wins: [(w[0], w[2]) for w in wins]) if ndim == 2 else (lambda wins: wins)
    v = np.array([float(x) for x in second_derivative_weights(order)], dtype=np.float64)
    w = np.array([0.0] + [float(x) for x in first_derivative_weights(order)], dtype=np.float64)
    pb = Problem(ndim, shape, tuple(float(h) for h in spacing), order // 2, v,
                 [(bc[2 * k], bc[2 * k + 1]) for k in range(ndim)], vel, vel * vel * dt * dt,
                 1.0 / (1.0 + e), e, float(dt), drop_y(sw), drop_y(rw), float(np.prod(spacing)), w)
    if rho is not None:
        pb.rho = np.asarray(rho, dtype=np.float64).reshape(shape)
        lr = np.log(pb.rho)
        pb.G = [first_deriv(lr, pb, ax, even=True) for ax in range(ndim)]
    return pb


def _ghosted(f: np.ndarray, pb: Problem, even: bool = False) -> np.ndarray:
    """f with R ghost nodes on every face, filled by the face conditions (or,
    with `even`, by the even mirror on every face)."""
    R = pb.R
    g = np.pad(f, R)
    for ax in range(pb.ndim):
        lo, hi = (BC_NEUMANN, BC_NEUMANN) if even else pb.bc[ax]
        n = f.shape[ax]
        for j in range(1, R + 1):
            for side, kind in ((0, lo), (1, hi)):
                ghost = R - j if side == 0 else R + n - 1 + j
                mirror = R + j if side == 0 else R + n - 1 - j
                dst = [slice(None)] * pb.ndim
                src = [slice(None)] * pb.ndim
                dst[ax] = ghost
                src[ax] = mirror
                if kind == BC_DIRICHLET:
                    g[tuple(dst)] = -g[tuple(src)]
                elif kind == BC_NEUMANN:
                    g[tuple(dst)] = g[tuple(src)]
                else:
                    g[tuple(dst)] = 0.0
    return g


def laplacian(f: np.ndarray, pb: Problem) -> np.ndarray:
    """Eq. 9 on node values with face-condition ghosts (oracle.c's operator)."""
    R = pb.R
    g = _ghosted(f, pb)
    out = np.zeros_like(f)
    core = tuple(slice(R, R + n) for n in f.shape)
    for ax in range(pb.ndim):
        h2 = pb.spacing[ax] ** 2
        acc = pb.v[0] * g[core]
        for j in range(1, R + 1):
            up = list(core)
            dn = list(core)
            up[ax] = slice(R + j, R + j + f.shape[ax])
            dn[ax] = slice(R - j, R - j + f.shape[ax])
            acc = acc + pb.v[j] * (g[tuple(up)] + g[tuple(dn)])
        out += acc / h2
    return out


def laplacian_t(f: np.ndarray, pb: Problem) -> np.ndarray:
    """Transpose of laplacian(): the same gather, corrected along Neumann faces
    (+ v_k / h^2 f_face at distance k = 1..R, - sum_j v_j / h^2 f_j at the face)."""
    out = laplacian(f, pb)
    for ax in range(pb.ndim):
        h2 = pb.spacing[ax] ** 2
        n = f.shape[ax]
        for side, kind in enumerate(pb.bc[ax]):
            if kind != BC_NEUMANN:
                continue
            def at(k):  # index tuple of the plane k nodes in from this face
                idx = [slice(None)] * pb.ndim
                idx[ax] = k if side == 0 else n - 1 - k
                return tuple(idx)
            fv = f[at(0)].copy()
            for k in range(1, pb.R + 1):
                out[at(k)] += pb.v[k] / h2 * fv
                out[at(0)] -= pb.v[k] / h2 * f[at(k)]
    return out


def first_deriv(f: np.ndarray, pb: Problem, ax: int, even: bool = False) -> np.ndarray:
    """Eq. 10 along axis ax: (1/2h) sum_j w_j (f[+j] - f[-j]) on ghosted node values."""
    R = pb.R
    g = _ghosted(f, pb, even)
    core = tuple(slice(R, R + n) for n in f.shape)
    out = np.zeros_like(f)
    for j in range(1, R + 1):
        up = list(core)
        dn = list(core)
        up[ax] = slice(R + j, R + j + f.shape[ax])
        dn[ax] = slice(R - j, R - j + f.shape[ax])
        out += pb.w[j] * (g[tuple(up)] - g[tuple(dn)])
    return out / (2.0 * pb.spacing[ax])


def first_deriv_t(q: np.ndarray, pb: Problem, ax: int, even: bool = False) -> np.ndarray:
    """Transpose of first_deriv: scatter each node's weights onto the ghosted
    array, then fold every ghost onto the node it mirrors (with its sign)."""
    R = pb.R
    n = q.shape[ax]
    ext = np.zeros(tuple(s + 2 * R for s in q.shape))
    core = tuple(slice(R, R + s) for s in q.shape)
    for j in range(1, R + 1):
        up = list(core)
        dn = list(core)
        up[ax] = slice(R + j, R + j + n)
        dn[ax] = slice(R - j, R - j + n)
        ext[tuple(up)] += pb.w[j] * q
        ext[tuple(dn)] -= pb.w[j] * q
    ext /= 2.0 * pb.spacing[ax]
    lo, hi = (BC_NEUMANN, BC_NEUMANN) if even else pb.bc[ax]
    for side, kind in ((0, lo), (1, hi)):
        if kind == BC_NONE:
            continue
        sign = -1.0 if kind == BC_DIRICHLET else 1.0
        for m in range(1, R + 1):
            src = [slice(None)] * q.ndim
            dst = [slice(None)] * q.ndim
            src[ax] = R - m if side == 0 else R + n - 1 + m   # the ghost
            dst[ax] = R + m if side == 0 else R + n - 1 - m   # the node it mirrors
            ext[tuple(dst)] += sign * ext[tuple(src)]
    return ext[core]


def operator(f: np.ndarray, pb: Problem) -> np.ndarray:
    """The spatial operator of the forward step: L, or L_rho with density."""
    out = laplacian(f, pb)
    if pb.rho is not None:
        for ax in range(pb.ndim):
            out -= pb.G[ax] * first_deriv(f, pb, ax)
    return out


def operator_t(q: np.ndarray, pb: Problem) -> np.ndarray:
    """Transpose of operator()."""
    out = laplacian_t(q, pb)
    if pb.rho is not None:
        for ax in range(pb.ndim):
            out -= first_deriv_t(pb.G[ax] * q, pb, ax)
    return out


def _zero_dirichlet(f: np.ndarray, pb: Problem) -> None:
    for ax in range(pb.ndim):
        for side, kind in enumerate(pb.bc[ax]):
            if kind == BC_DIRICHLET:
                idx = [slice(None)] * pb.ndim
                idx[ax] = 0 if side == 0 else f.shape[ax] - 1
                f[tuple(idx)] = 0.0


def _window_field(win, shape, scale=1.0) -> np.ndarray:
    """Dense field of a separable window (first node and weights per axis)."""
    out = np.zeros(shape)
    idx = tuple(slice(f, f + len(w)) for f, w in win)
    block = np.ones([len(w) for _, w in win])
    for ax, (_, w) in enumerate(win):
        sh = [1] * len(win)
        sh[ax] = len(w)
        block = block * np.asarray(w, dtype=np.float64).reshape(sh)
    out[idx] = block * scale
    return out


def source_fields(pb: Problem) -> List[np.ndarray]:
    """Per source: window weights / prod(h) as a dense field (s[n] = sum S_s(t_n) field_s)."""
    return [_window_field(w, pb.shape, 1.0 / pb.cell) for w in pb.src]


def receiver_fields(pb: Problem) -> List[np.ndarray]:
    return [_window_field(w, pb.shape) for w in pb.rec]


def forward_states(pb: Problem, wavelet: np.ndarray, n_steps: int):
    """Every p[n] (n = 0 .. N) and the seismogram [N][n_rec]."""
    wav = np.asarray(wavelet, dtype=np.float64)
    wav = np.broadcast_to(wav, (len(pb.src), wav.shape[-1])) if len(pb.src) else wav
    sf, rf = source_fields(pb), receiver_fields(pb)
    p_prev = np.zeros(pb.shape)
    p = np.zeros(pb.shape)
    states = [p.copy()]
    seis = np.zeros((n_steps, len(rf)))
    for n in range(n_steps):
        s = sum((wav[i, n] * sf[i] for i in range(len(sf))), np.zeros(pb.shape))
        nxt = pb.a * (2.0 * p + pb.kappa * operator(p, pb) - (1.0 - pb.e) * p_prev) + pb.a * pb.kappa * s
        _zero_dirichlet(nxt, pb)
        p_prev, p = p, nxt
        states.append(p.copy())
        seis[n] = [float(np.sum(r * p)) for r in rf]
    return states, seis


def backward(pb: Problem, residual: np.ndarray, n_steps: int, states=None, wavelet=None):
    """The adjoint sweep for a given residual [N][n_rec].  Returns (dJ/dc or
    None, adjoint source trace [n_src][N]); the gradient needs the forward
    states p[0..N] and the wavelet.  backward_full also returns dJ/drho.

    The adjoint source trace dJ/dS_s(t_n) = sum_k (source weights / prod h)_k
    psi[n+1]_k is the transpose of the wavelet-to-seismogram map applied to
    the residual.
    """
    g_c, _, adj_src = backward_full(pb, residual, n_steps, states, wavelet)
    return g_c, adj_src


def backward_full(pb: Problem, residual: np.ndarray, n_steps: int, states=None, wavelet=None):
    """(dJ/dc or None, dJ/drho or None, adjoint source trace [n_src][N])."""
    res = np.asarray(residual, dtype=np.float64)
    sf, rf = source_fields(pb), receiver_fields(pb)
    if wavelet is not None and len(sf):
        wav = np.broadcast_to(np.asarray(wavelet, dtype=np.float64), (len(sf), np.shape(wavelet)[-1]))
    g_kappa = np.zeros(pb.shape) if states is not None else None
    g_G = [np.zeros(pb.shape) for _ in range(pb.ndim)] if states is not None and pb.rho is not None else None
    adj_src = np.zeros((len(sf), n_steps))
    psi1 = np.zeros(pb.shape)  # psi[k+1]
    psi2 = np.zeros(pb.shape)  # psi[k+2]
    for k in range(n_steps, 0, -1):
        rt = sum((res[k - 1, i] * rf[i] for i in range(len(rf))), np.zeros(pb.shape))
        psi = pb.a * (2.0 * psi1 + pb.kappa * operator_t(psi1, pb) - (1.0 - pb.e) * psi2) + pb.kappa * pb.a * rt
        _zero_dirichlet(psi, pb)
        n = k - 1  # psi[k] pairs with p[k-1]: dp[k]/dkappa = Z a (L p[k-1] + s[k-1])
        if states is not None:
            s = sum((wav[i, n] * sf[i] for i in range(len(sf))), np.zeros(pb.shape))
            g_kappa += psi * (operator(states[n], pb) + s) / pb.kappa
            if g_G is not None:  # d p[k] / d G_a = - Z a kappa D_a p[k-1]
                for ax in range(pb.ndim):
                    g_G[ax] -= psi * first_deriv(states[n], pb, ax)
        for i in range(len(sf)):
            adj_src[i, n] = float(np.sum(sf[i] * psi))
        psi2, psi1 = psi1, psi
    g_c = None if g_kappa is None else 2.0 * pb.vel * pb.dt * pb.dt * g_kappa
    g_rho = None
    if g_G is not None:
        g_lnrho = sum(first_deriv_t(g_G[ax], pb, ax, even=True) for ax in range(pb.ndim))
        g_rho = g_lnrho / pb.rho
    return g_c, g_rho, adj_src


def adjoint_gradient(pb: Problem, wavelet: np.ndarray, observed: np.ndarray, n_steps: int):
    """(misfit J, dJ/dc on the nodes, adjoint source trace [n_src][N])."""
    states, seis = forward_states(pb, wavelet, n_steps)
    res = seis - np.asarray(observed, dtype=np.float64)[:n_steps]
    J = 0.5 * float(np.sum(res * res))
    g_c, adj_src = backward(pb, res, n_steps, states, wavelet)
    return J, g_c, adj_src


def adjoint_gradient_full(pb: Problem, wavelet: np.ndarray, observed: np.ndarray, n_steps: int):
    """(misfit J, dJ/dc, dJ/drho (None for constant density), adjoint source trace)."""
    states, seis = forward_states(pb, wavelet, n_steps)
    res = seis - np.asarray(observed, dtype=np.float64)[:n_steps]
    J = 0.5 * float(np.sum(res * res))
    g_c, g_rho, adj_src = backward_full(pb, res, n_steps, states, wavelet)
    return J, g_c, g_rho, adj_src
