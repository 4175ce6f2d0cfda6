"""Python binding of the C ABI (include/simwave_b300.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays may be
torch tensors (CPU or CUDA) or numpy arrays; they must be contiguous FP32 for
grid-shaped data.  Each failing call raises SimwaveError with the library's
status and message.  All computation happens in the CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib

SW_OK, SW_EINVAL, SW_ECFL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT, SW_ESTATE = range(7)
SW_BC_NONE, SW_BC_DIRICHLET, SW_BC_NEUMANN = 0, 1, 2
SW_STENCIL_AUTO, SW_STENCIL_PLAIN, SW_STENCIL_TMA, SW_STENCIL_CLUSTER, SW_STENCIL_TB2 = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "SW_OK", 1: "SW_EINVAL", 2: "SW_ECFL", 3: "SW_ENOMEM", 4: "SW_ECUDA",
                5: "SW_ETIMEOUT", 6: "SW_ESTATE"}
BC_NAMES = {"none": SW_BC_NONE, "null_dirichlet": SW_BC_DIRICHLET, "dirichlet": SW_BC_DIRICHLET,
            "null_neumann": SW_BC_NEUMANN, "neumann": SW_BC_NEUMANN}


class SimwaveError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


def _check(status: int):
    if status != SW_OK:
        msg = _lib.load().sw_last_error()
        raise SimwaveError(status, msg.decode() if msg else "")


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") and callable(a.numel) else int(np.asarray(a).size)


def _need(name: str, a, n: int, at_least: bool = False) -> None:
    """Raises ValueError unless the buffer `a` (if given) holds n values (at
    least n with at_least): the C calls read and write whole buffers of the
    sizes the grid implies and cannot see the caller's."""
    if a is None:
        return
    k = _numel(a)
    if (k < n) if at_least else (k != n):
        raise ValueError("%s holds %d values, needs %s%d" % (name, k, ">= " if at_least else "", n))


def _ptr(a) -> Optional[int]:
    """Raw address of a contiguous FP32 tensor / array (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("expected a contiguous float32 tensor")
        return a.data_ptr()
    arr = np.asarray(a)
    if arr.dtype != np.float32 or not arr.flags.c_contiguous:
        raise ValueError("expected a C-contiguous float32 array")
    return arr.ctypes.data


class Grid:
    """Owner of an sw_grid handle; destroyed with sw_destroy_grid."""

    def __init__(self, handle: int, ndim: int, shape, stream):
        self.handle = handle
        self.ndim = ndim
        self.shape = tuple(int(s) for s in shape)
        self.stream = stream
        self.n_src = 0
        self.n_rec = 0
        self._keep = []

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            _lib.load().sw_destroy_grid(self.handle)
            self.handle = None


def _faces(vals, ndim, names=None):
    vals = list(vals)
    if len(vals) != 2 * ndim:
        raise ValueError("expected %d face values" % (2 * ndim))
    if names:
        vals = [names[v] if isinstance(v, str) else int(v) for v in vals]
    return (ctypes.c_int * len(vals))(*vals)


def sw_create_grid(ndim: int, shape: Sequence[int], spacing: Sequence[float], space_order: int,
                   nbl: Sequence[int], bc: Sequence, damp_alpha: float = 0.0, damp_degree: int = 3,
                   dt: float = 0.0, stream=None) -> Grid:
    lib = _lib.load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * ndim)(*[int(s) for s in shape])
    spc = (ctypes.c_double * ndim)(*[float(s) for s in spacing])
    _check(lib.sw_create_grid(ctypes.byref(h), int(ndim), shp, spc, int(space_order),
                              _faces(nbl, ndim), _faces(bc, ndim, BC_NAMES), float(damp_alpha),
                              int(damp_degree), float(dt), ctypes.c_void_p(stream)))
    return Grid(h.value, ndim, shape, stream)


def sw_set_model(g: Grid, velocity, density=None) -> None:
    _need("velocity", velocity, g.nodes)
    _need("density", density, g.nodes)
    _check(_lib.load().sw_set_model(g.handle, _ptr(velocity), _ptr(density)))


def sw_set_acquisition(g: Grid, src_pos, rec_pos, wavelet, window_radius: int = 4,
                       wavelet_per_source: bool = False) -> None:
    src = np.ascontiguousarray(np.asarray(src_pos, dtype=np.float64).reshape(-1, g.ndim))
    rec = np.ascontiguousarray(np.asarray(rec_pos, dtype=np.float64).reshape(-1, g.ndim))
    if hasattr(wavelet, "data_ptr"):
        wav = wavelet
        nt = int(wavelet.shape[-1])
    else:
        wav = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float32))
        nt = int(wav.shape[-1])
    # the library reads n_src * nt samples with one wavelet per source, nt otherwise
    _need("wavelet", wav, (int(src.shape[0]) if wavelet_per_source else 1) * nt, at_least=True)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_lib.load().sw_set_acquisition(
        g.handle, int(src.shape[0]), src.ctypes.data_as(dp), int(rec.shape[0]), rec.ctypes.data_as(dp),
        nt, _ptr(wav), int(bool(wavelet_per_source)), int(window_radius)))
    g.n_src = int(src.shape[0])
    g.n_rec = int(rec.shape[0])
    g._keep = [wav]


def sw_forward(g: Grid, n_steps: int, seismogram=None, final_field=None) -> None:
    """Runs n_steps steps; writes into the given output tensors/arrays (either may be None)."""
    _need("seismogram", seismogram, max(int(n_steps), 0) * g.n_rec, at_least=True)
    _need("final_field", final_field, g.nodes)
    _check(_lib.load().sw_forward(g.handle, int(n_steps), _ptr(seismogram), _ptr(final_field)))


SW_CKPT_FP32, SW_CKPT_BF16, SW_CKPT_FP16, SW_CKPT_I16 = 0, 1, 2, 3


def sw_gradient(g: Grid, n_steps: int, observed, grad_vel, checkpoint_every: int = 0,
                checkpoint_format: int = SW_CKPT_FP32, grad_rho=None) -> float:
    """Misfit J = 1/2 |d - observed|^2 of a forward run, dJ/dvelocity into
    grad_vel and (density models) dJ/ddensity into grad_rho (adjoint-state
    method); returns J."""
    _need("observed", observed, max(int(n_steps), 0) * g.n_rec, at_least=True)
    _need("grad_vel", grad_vel, g.nodes)
    _need("grad_rho", grad_rho, g.nodes)
    j = ctypes.c_double()
    _check(_lib.load().sw_gradient(g.handle, int(n_steps), _ptr(observed), ctypes.byref(j), _ptr(grad_vel),
                                   _ptr(grad_rho), int(checkpoint_every), int(checkpoint_format)))
    return j.value


def sw_gradient_shots(g: Grid, shot_src_pos, n_steps: int, observed, grad_vel, checkpoint_every: int = 0,
                      checkpoint_format: int = SW_CKPT_FP32, grad_rho=None) -> float:
    """Misfit and gradient summed over shots: shot s moves the acquisition's
    sources to shot_src_pos[s] ([n_shots][n_src][ndim] or [n_shots][ndim] for
    one source per shot, metres) and is compared with observed[s]
    ([n_shots][n_steps][n_rec]); returns sum_s J_s, writes sum_s dJ_s/dc into
    grad_vel (and sum_s dJ_s/drho into grad_rho)."""
    pos = np.ascontiguousarray(np.asarray(shot_src_pos, dtype=np.float64))
    n_shots = int(pos.shape[0])
    if n_shots < 1 or pos.size % (n_shots * g.ndim) != 0:
        raise ValueError("shot_src_pos must be [n_shots][n_src][ndim]")
    if pos.size != n_shots * g.n_src * g.ndim:
        raise ValueError("shot_src_pos holds %d values, needs n_shots x n_src x ndim = %d"
                         % (pos.size, n_shots * g.n_src * g.ndim))
    if int(np.prod(observed.shape)) != n_shots * int(n_steps) * g.n_rec:
        raise ValueError("observed must hold [n_shots][n_steps][n_rec] = %d values" % (n_shots * n_steps * g.n_rec))
    _need("grad_vel", grad_vel, g.nodes)
    _need("grad_rho", grad_rho, g.nodes)
    j = ctypes.c_double()
    _check(_lib.load().sw_gradient_shots(g.handle, n_shots, pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(n_steps), _ptr(observed), ctypes.byref(j), _ptr(grad_vel),
                                         _ptr(grad_rho), int(checkpoint_every), int(checkpoint_format)))
    return j.value


def _f32(a):
    """A contiguous FP32 view of a tensor or array (tensors pass through)."""
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def sw_set_forcing(g: Grid, fields=None, signatures=None) -> None:
    """Distributed forcing sum_m F_m(x) T_m(t_n): fields [n_force, *grid], signatures
    [n_force, n_sig] (host or device, copied).  None removes the forcing."""
    if fields is None:
        _check(_lib.load().sw_set_forcing(g.handle, 0, None, None, 0))
        return
    F, T = _f32(fields), _f32(signatures)
    n_force = int(F.shape[0])
    if tuple(F.shape[1:]) != g.shape or T.ndim != 2 or int(T.shape[0]) != n_force:
        raise ValueError("expected fields [n_force, *grid] and signatures [n_force, n_sig]")
    _check(_lib.load().sw_set_forcing(g.handle, n_force, _ptr(F), _ptr(T), int(T.shape[1])))


def sw_set_initial_state(g: Grid, p0=None, pm1=None) -> None:
    """Initial levels p[0], p[-1] of later forwards (grid-shaped; None = zero)."""
    a, b = _f32(p0), _f32(pm1)
    for x in (a, b):
        if x is not None and tuple(x.shape) != g.shape:
            raise ValueError("expected a field of the grid's shape")
    _check(_lib.load().sw_set_initial_state(g.handle, _ptr(a), _ptr(b)))


def sw_set_saving(g: Grid, saving_stride: int, snapshots=None, max_frames: int = 0) -> None:
    """Every later sw_forward writes p after saving_stride, 2 saving_stride, ...
    steps into the frames of `snapshots` (device, [max_frames, *grid]); 0 turns it off."""
    _need("snapshots", snapshots, max(int(max_frames), 0) * g.nodes, at_least=True)
    _check(_lib.load().sw_set_saving(g.handle, int(saving_stride), _ptr(snapshots), int(max_frames)))


class Batch:
    """Owner of an sw_batch handle (destroyed with sw_destroy_batch); keeps its grids alive."""

    def __init__(self, handle: int, grids):
        self.handle = handle
        self.grids = list(grids)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            _lib.load().sw_destroy_batch(self.handle)
            self.handle = None


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, a in enumerate(items):
        arr[i] = _ptr(a)
    return arr


def sw_create_batch(grids) -> Batch:
    """Batch of constant-density grids advanced together: 2D grids (shots of one model share its reads) or 3D
    grids (one pipelined stencil launch and one face launch per step for all)."""
    grids = list(grids)
    handles = (ctypes.c_void_p * len(grids))(*[g.handle for g in grids])
    h = ctypes.c_void_p()
    _check(_lib.load().sw_create_batch(ctypes.byref(h), handles, len(grids)))
    return Batch(h.value, grids)


def sw_batch_forward(b: Batch, n_steps: int, seismograms=None, final_fields=None) -> None:
    """seismograms: per grid a device tensor [n_steps, n_rec] (or None); final_fields: per grid or None."""
    n = len(b.grids)
    seismograms = list(seismograms) if seismograms is not None else [None] * n
    if len(seismograms) != n or (final_fields is not None and len(list(final_fields)) != n):
        raise ValueError("expected one seismogram (or None) and one final field per grid (%d)" % n)
    for i, (g, s_) in enumerate(zip(b.grids, seismograms)):
        _need("seismogram of grid %d" % i, s_, max(int(n_steps), 0) * g.n_rec, at_least=True)
    if final_fields is not None:
        final_fields = list(final_fields)
        for i, (g, f_) in enumerate(zip(b.grids, final_fields)):
            _need("final field of grid %d" % i, f_, g.nodes)
    seis = _ptr_array(seismograms)
    fin = _ptr_array(final_fields) if final_fields is not None else None
    _check(_lib.load().sw_batch_forward(b.handle, int(n_steps), seis, fin))


def sw_batch_info(b: Batch):
    """(model groups, work items per step: tiles x shots)."""
    ng, nt = ctypes.c_int(), ctypes.c_int()
    _check(_lib.load().sw_batch_info(b.handle, ctypes.byref(ng), ctypes.byref(nt)))
    return ng.value, nt.value


def sw_batch_get_tile(b: Batch):
    """(tile height in use, [us per stencil launch with heights 16, 32, 64] as timed by the tuner)."""
    rows = ctypes.c_int()
    us = (ctypes.c_float * 3)()
    _check(_lib.load().sw_batch_get_tile(b.handle, ctypes.byref(rows), us))
    return rows.value, list(us)


def sw_batch_set_tile(b: Batch, tile_rows: int) -> None:
    """Force the tile height (16, 32 or 64 rows) instead of the tuner's choice."""
    _check(_lib.load().sw_batch_set_tile(b.handle, int(tile_rows)))


def sw_batch_set_profiling(b: Batch, every=1) -> None:
    _check(_lib.load().sw_batch_set_profiling(b.handle, int(every)))


def sw_batch_get_profile(b: Batch):
    """(summed ms of the timed stencil launches, timed launches, kernel launches) of the last batch forward."""
    ms = ctypes.c_double()
    n1 = ctypes.c_int64()
    n2 = ctypes.c_int64()
    _check(_lib.load().sw_batch_get_profile(b.handle, ctypes.byref(ms), ctypes.byref(n1), ctypes.byref(n2)))
    return ms.value, n1.value, n2.value


def sw_set_checkpoint_budget(g: Grid, max_states: int) -> None:
    """sw_gradient keeps at most max_states forward states (binomial schedule); 0: uniform segments."""
    _check(_lib.load().sw_set_checkpoint_budget(g.handle, int(max_states)))


def sw_get_dt(g: Grid) -> float:
    v = ctypes.c_double()
    _check(_lib.load().sw_get_dt(g.handle, ctypes.byref(v)))
    return v.value


def sw_ricker(f_peak: float, t0: float, dt: float, nt: int) -> np.ndarray:
    out = np.zeros(int(nt), dtype=np.float32)
    _check(_lib.load().sw_ricker(float(f_peak), float(t0), float(dt), int(nt), out.ctypes.data))
    return out


def sw_set_pipeline_test(g: Grid, starve: bool, wait_limit_ns: int = 0) -> None:
    """Failure-path test hook: with `starve` the pipelined kernel issues no
    copies, so its bounded waits give up and sw_forward raises SW_ETIMEOUT."""
    _check(_lib.load().sw_set_pipeline_test(g.handle, int(bool(starve)), int(wait_limit_ns)))


def sw_set_stencil_variant(g: Grid, variant: int) -> None:
    _check(_lib.load().sw_set_stencil_variant(g.handle, int(variant)))


def sw_get_stencil_variant(g: Grid) -> int:
    v = ctypes.c_int()
    _check(_lib.load().sw_get_stencil_variant(g.handle, ctypes.byref(v)))
    return v.value


def sw_set_profiling(g: Grid, every=1) -> None:
    """Time every `every`-th stencil launch of sw_forward (True: all, False/0: none)."""
    _check(_lib.load().sw_set_profiling(g.handle, int(every)))


def sw_get_profile(g: Grid):
    """(summed ms of the timed stencil launches, timed launches, kernel launches) of the last sw_forward."""
    ms = ctypes.c_double()
    n1 = ctypes.c_int64()
    n2 = ctypes.c_int64()
    _check(_lib.load().sw_get_profile(g.handle, ctypes.byref(ms), ctypes.byref(n1), ctypes.byref(n2)))
    return ms.value, n1.value, n2.value


def sw_get_device_bytes(g: Grid) -> int:
    v = ctypes.c_int64()
    _check(_lib.load().sw_get_device_bytes(g.handle, ctypes.byref(v)))
    return v.value


SW_NOALLOC_SCRATCH_BYTES = 32 << 20


def sw_forward_noalloc(ndim: int, shape: Sequence[int], spacing: Sequence[float], space_order: int,
                       nbl: Sequence[int], bc: Sequence, damp_alpha: float, damp_degree: int, dt: float,
                       velocity, density, src_pos, rec_pos, wavelet, window_radius: int, n_steps: int,
                       seismogram=None, final_field=None, wavelet_per_source: bool = False, stream=None) -> None:
    """Forward run that allocates no device memory (see sw_forward_noalloc in the C header).

    velocity / density / seismogram / final_field must be CUDA tensors on the
    current device; the outputs must be preallocated by the caller.  The sizes
    are checked here against shape, the source and receiver counts and
    n_steps before the call (the C entry point only sees raw pointers).
    """
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    src = np.ascontiguousarray(np.asarray(src_pos, dtype=np.float64).reshape(-1, ndim))
    rec = np.ascontiguousarray(np.asarray(rec_pos, dtype=np.float64).reshape(-1, ndim))
    if hasattr(wavelet, "data_ptr"):
        wav = wavelet
    else:
        wav = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float32))
    nt = int(wav.shape[-1]) if wav.ndim else 1
    n_src, n_rec = int(src.shape[0]), int(rec.shape[0])
    nodes = int(np.prod([int(s) for s in shape]))
    here = torch.cuda.current_device()

    def on_device(name, t, numel, at_least=False):
        if t is None:
            return
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.device.index == here):
            raise ValueError("%s must be a CUDA tensor on the current device (cuda:%d)" % (name, here))
        if (t.numel() < numel) if at_least else (t.numel() != numel):
            raise ValueError("%s holds %d values, needs %s%d" % (name, t.numel(), ">= " if at_least else "", numel))

    on_device("velocity", velocity, nodes)
    on_device("density", density, nodes)
    on_device("final_field", final_field, nodes)
    if n_rec > 0 and n_steps > 0:
        if seismogram is None:
            raise ValueError("seismogram is needed with receivers")
        on_device("seismogram", seismogram, int(n_steps) * n_rec, at_least=True)
    if n_src > 0:
        want = n_src * nt if wavelet_per_source else nt
        if int(np.prod(wav.shape)) != want:
            raise ValueError("wavelet holds %d samples, needs %d" % (int(np.prod(wav.shape)), want))
        if hasattr(wav, "is_cuda") and wav.is_cuda and wav.device.index != here:
            raise ValueError("the wavelet is on another device than the current one")
    dp = ctypes.POINTER(ctypes.c_double)
    shp = (ctypes.c_int64 * ndim)(*[int(s) for s in shape])
    spc = (ctypes.c_double * ndim)(*[float(s) for s in spacing])
    _check(_lib.load().sw_forward_noalloc(
        int(ndim), shp, spc, int(space_order), _faces(nbl, ndim), _faces(bc, ndim, BC_NAMES), float(damp_alpha),
        int(damp_degree), float(dt), _ptr(velocity), _ptr(density), n_src, src.ctypes.data_as(dp),
        n_rec, rec.ctypes.data_as(dp), nt, _ptr(wav), int(bool(wavelet_per_source)),
        int(window_radius), int(n_steps), _ptr(seismogram), _ptr(final_field), ctypes.c_void_p(stream)))


def sw_last_error() -> str:
    msg = _lib.load().sw_last_error()
    return msg.decode() if msg else ""


def sw_destroy_grid(g: Grid) -> None:
    g.close()
