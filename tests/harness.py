"""Run one workload through the CUDA library (C ABI) and through the FP64 oracle.

Test-side glue only: the GPU run goes through paper_2201_05278_b300.api (the
C ABI), the reference run through oracle.forward; both read the same
workload description from paper_2201_05278_b300.workloads.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_2201_05278_b300 import api
from paper_2201_05278_b300.workloads import Workload

FP32_SEIS_TOL = 1e-5  # relative L2 on the seismogram, FP32 forward vs FP64 oracle
# Element-wise bar: every sample / node within this fraction of the largest
# magnitude of the reference, so that an error confined to a few nodes (a wrong
# face row, a stale halo, a ragged tile edge) cannot hide under the global norm.
FP32_MAX_TOL = 1e-5


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def max_rel(a, b) -> float:
    """max |a - b| / max |b| (max |a - b| when b is all zero)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0 and b.size == 0:
        return 0.0
    d = float(np.abs(a - b).max())
    mb = float(np.abs(b).max())
    return d / mb if mb > 0 else d


def _log_parity(what, e2, einf):
    path = os.environ.get("PARITY_LOG")
    if not path:
        return
    import json
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, "what": what, "rel_l2": e2, "max_rel": einf}) + "\n")


def parity(a, b, what=""):
    """(relative L2, element-wise max relative) of a against the reference b, logged
    to $PARITY_LOG when set."""
    e2, einf = rel_l2(a, b), max_rel(a, b)
    _log_parity(what, e2, einf)
    return e2, einf


def assert_parity(a, b, what="", tol=FP32_SEIS_TOL, max_tol=FP32_MAX_TOL):
    """Both bars: relative L2 <= tol and every element within max_tol * max|b|."""
    e2, einf = parity(a, b, what)
    assert e2 <= tol and einf <= max_tol, "%s: rel-L2 %.3e (bar %.0e), max %.3e of peak (bar %.0e)" % (
        what or "parity", e2, tol, einf, max_tol)


def wavelet_of(w: Workload, nt=None):
    return oracle.ricker_samples(w.f_peak, w.dt, nt or w.n_steps, t0=w.t0)


def run_gpu(w: Workload, n_steps=None, device_io=True, wavelet=None, final=True, profile=False, variant=None,
            expect_variant=None):
    import torch
    n_steps = w.n_steps if n_steps is None else n_steps
    dev = torch.device("cuda:0")
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree,
                           w.dt)
    try:
        vel = torch.from_numpy(np.ascontiguousarray(w.velocity, dtype=np.float32))
        rho = None if w.density is None else torch.from_numpy(np.ascontiguousarray(w.density, np.float32))
        if device_io:
            vel = vel.to(dev)
            rho = None if rho is None else rho.to(dev)
        api.sw_set_model(g, vel, rho)
        if variant is not None:
            api.sw_set_stencil_variant(g, variant)
        if expect_variant is not None:
            assert api.sw_get_stencil_variant(g) == expect_variant
        if wavelet is None:
            wavelet = api.sw_ricker(w.f_peak, w.t0, w.dt, max(n_steps, 1))
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wavelet, window_radius=w.window_radius)
        if profile:
            api.sw_set_profiling(g, True)
        n_rec = len(w.rec_pos)
        if device_io:
            seis = torch.zeros((n_steps, n_rec), dtype=torch.float32, device=dev)
            fin = torch.zeros(w.shape, dtype=torch.float32, device=dev) if final else None
        else:
            seis = np.zeros((n_steps, n_rec), dtype=np.float32)
            fin = np.zeros(w.shape, dtype=np.float32) if final else None
        api.sw_forward(g, n_steps, seis if n_rec else None, fin)
        prof = api.sw_get_profile(g) if profile else None
        if device_io:
            seis = seis.cpu().numpy()
            fin = fin.cpu().numpy() if final else None
        return (seis, fin, prof) if profile else (seis, fin)
    finally:
        g.close()


def run_oracle(w: Workload, n_steps=None, wavelet=None, threads=0):
    n_steps = w.n_steps if n_steps is None else n_steps
    if wavelet is None:
        wavelet = wavelet_of(w, max(n_steps, 1))
    return oracle.forward(w.ndim, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt, n_steps,
                          src_pos=[tuple(p) for p in w.src_pos], wavelet=np.asarray(wavelet, np.float64),
                          rec_pos=[tuple(p) for p in w.rec_pos], nbl=w.nbl, bc=w.bc,
                          damp_alpha=w.damp_alpha, damp_degree=w.damp_degree,
                          rho=None if w.density is None else w.density.astype(np.float64),
                          window_radius=w.window_radius, threads=threads or os.cpu_count())
