"""High-level FP64 oracle forward: builds the setup, calls oracle.c.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

forward() follows the order of the paper's solver (Sec. 2.1-2.4, Sec. 3-4):
FD weights (Eq. 9-10), damping profile (Eq. 4), kappa = c^2 dt^2, ln(rho) for
variable density (Eq. 5), Kaiser-sinc windows (Eq. 11-12), then the leapfrog
loop of Eq. 7 in oracle.c.  Every array is FP64.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from .damping import eta_field
from .fd import first_derivative_weights, second_derivative_weights
from .source import KAISER_B, point_windows

BC_NONE, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
_BC_NAMES = {"none": BC_NONE, "null_dirichlet": BC_DIRICHLET, "dirichlet": BC_DIRICHLET,
             "null_neumann": BC_NEUMANN, "neumann": BC_NEUMANN}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_forward.restype = ctypes.c_int
        lib.oracle_forward.argtypes = [
            ctypes.c_int, i64, d, ctypes.c_int, d, d, ip, d, ctypes.c_double, d, d,
            ctypes.c_int, i64, ip, ctypes.c_int, d, d, ctypes.c_int,
            ctypes.c_int, i64, ip, ctypes.c_int, d,
            ctypes.c_int, d, d, d, d,
            ctypes.c_int, d, d, d, ctypes.c_int]
        _lib = lib
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _bc_codes(bc) -> list:
    return [b if isinstance(b, int) else _BC_NAMES[b] for b in bc]


def _pack_windows(wins):
    n = len(wins)
    lens = [len(wins[0][a][1]) for a in range(3)] if n else [1, 1, 1]
    lmax = max(lens)
    first = np.zeros((max(n, 1), 3), dtype=np.int64)
    w = np.zeros((max(n, 1), 3, lmax), dtype=np.float64)
    for i, axes in enumerate(wins):
        for a in range(3):
            first[i, a] = axes[a][0]
            w[i, a, : len(axes[a][1])] = axes[a][1]
    return first, np.asarray(lens, dtype=np.int32), lmax, w


def run_raw(ndim, shape, spacing, order, bc, eta, dt, vel, lnrho=None,
            src_windows=(), src_sig=None, rec_windows=(), n_steps=0,
            force_fields=None, force_sigs=None, p0=None, pm1=None, threads=0,
            want_prev=False):
    """Call oracle_forward with prepared FP64 arrays.  Returns (seis, p_last[, p_prev])."""
    lib = _load()
    shape = tuple(int(s) for s in shape)
    grid = shape if ndim == 3 else shape
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(grid)
    eta = np.ascontiguousarray(eta, dtype=np.float64).reshape(grid)
    if lnrho is not None:
        lnrho = np.ascontiguousarray(lnrho, dtype=np.float64).reshape(grid)
    v = np.array([float(x) for x in second_derivative_weights(order)], dtype=np.float64)
    w = np.array([0.0] + [float(x) for x in first_derivative_weights(order)], dtype=np.float64)
    sf, sl, slmax, sw = _pack_windows(list(src_windows))
    rf, rl, rlmax, rw = _pack_windows(list(rec_windows))
    n_src, n_rec = len(src_windows), len(rec_windows)
    if n_src:
        src_sig = np.ascontiguousarray(src_sig, dtype=np.float64)
        if src_sig.ndim == 1:
            src_sig = np.ascontiguousarray(np.broadcast_to(src_sig, (n_src, src_sig.shape[0])))
        nt = src_sig.shape[1]
    else:
        src_sig = np.zeros((1, 1))
        nt = 0
    n_force = 0
    if force_fields is not None:
        force_fields = np.ascontiguousarray(force_fields, dtype=np.float64)
        force_sigs = np.ascontiguousarray(force_sigs, dtype=np.float64)
        n_force = force_fields.shape[0]
        assert force_sigs.shape == (n_force, n_steps)
    if p0 is not None:
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
    if pm1 is not None:
        pm1 = np.ascontiguousarray(pm1, dtype=np.float64)
    seis = np.zeros((n_steps, max(n_rec, 1)), dtype=np.float64)
    p_last = np.zeros(grid, dtype=np.float64)
    p_prev = np.zeros(grid, dtype=np.float64) if want_prev else None
    shape_arr = np.asarray(shape, dtype=np.int64)
    spacing_arr = np.asarray(spacing, dtype=np.float64)
    bc_arr = np.asarray(_bc_codes(bc), dtype=np.int32)
    if ndim == 2 and len(bc_arr) == 4:
        bc_arr = np.asarray([bc_arr[0], bc_arr[1], 0, 0, bc_arr[2], bc_arr[3]], dtype=np.int32)
    i64 = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib.oracle_forward(
        ndim, shape_arr.ctypes.data_as(i64), _dp(spacing_arr), order, _dp(v), _dp(w),
        bc_arr.ctypes.data_as(ip), _dp(eta), dt, _dp(vel), _dp(lnrho),
        n_src, sf.ctypes.data_as(i64), sl.ctypes.data_as(ip), slmax, _dp(sw), _dp(src_sig), nt,
        n_rec, rf.ctypes.data_as(i64), rl.ctypes.data_as(ip), rlmax, _dp(rw),
        n_force, _dp(force_fields), _dp(force_sigs), _dp(p0), _dp(pm1),
        n_steps, _dp(seis), _dp(p_last), _dp(p_prev), int(threads))
    if rc != 0:
        raise ValueError("oracle_forward failed with code %d" % rc)
    seis = seis[:, :n_rec]
    if want_prev:
        return seis, p_last, p_prev
    return seis, p_last


def forward(ndim: int, shape: Sequence[int], spacing: Sequence[float], order: int,
            vel: np.ndarray, dt: float, n_steps: int,
            src_pos: Sequence[Sequence[float]] = (), wavelet=None,
            rec_pos: Sequence[Sequence[float]] = (),
            nbl: Sequence[int] = None, bc: Sequence = None,
            damp_alpha: float = 0.0, damp_degree: int = 3,
            rho: Optional[np.ndarray] = None, window_radius: int = 4,
            kaiser_b: Optional[float] = None, threads: int = 0,
            force_fields=None, force_sigs=None, p0=None, pm1=None, want_prev=False):
    """FP64 forward simulation.

    shape, spacing, nbl (lo, hi per axis) and bc are in (z, [y,] x) order; shape
    includes the absorbing layer; positions are metres from the corner of the
    physical domain.  wavelet is [nt] (shared) or [n_src][nt].  Returns
    (seismogram [n_steps][n_rec], final field).
    """
    shape = tuple(int(s) for s in shape)
    if nbl is None:
        nbl = [0] * (2 * ndim)
    if bc is None:
        bc = [BC_DIRICHLET] * (2 * ndim)
    bc = _bc_codes(bc)
    if ndim == 2:
        bc6 = [bc[0], bc[1], BC_NONE, BC_NONE, bc[2], bc[3]]
    else:
        bc6 = list(bc)
    eta = eta_field(shape, nbl, damp_alpha, damp_degree)
    lnrho = None if rho is None else np.log(np.asarray(rho, dtype=np.float64))
    nbl_lo = [nbl[2 * a] for a in range(ndim)]
    b = kaiser_b if kaiser_b is not None else KAISER_B[window_radius]
    sw = point_windows(src_pos, ndim, spacing, nbl_lo, window_radius, b, shape)
    rw = point_windows(rec_pos, ndim, spacing, nbl_lo, window_radius, b, shape)
    return run_raw(ndim, shape, spacing, order, bc6, eta, dt, vel, lnrho,
                   sw, wavelet, rw, n_steps, force_fields, force_sigs, p0, pm1,
                   threads, want_prev)
