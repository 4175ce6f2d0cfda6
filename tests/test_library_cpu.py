"""Host-side checks of the CUDA library that need no GPU.

- the shared library loads and exports every function include/simwave_b300.h
  declares, and the Python binding knows each of them;
- the library's host set-up (Ricker samples) agrees with the oracle's;
- the seeded workload generators are deterministic and sized as documented.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2201_05278_b300 import _lib, api, build, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "simwave_b300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def test_library_ricker_matches_oracle(lib):
    out = api.sw_ricker(12.0, 0.09, 1e-3, 400)
    ref = np.array(oracle.ricker_samples(12.0, 1e-3, 400, t0=0.09))
    assert np.max(np.abs(out - ref)) < 1e-7


def test_library_rejects_bad_arguments_without_gpu(lib):
    with pytest.raises(api.SimwaveError):
        api.sw_ricker(-1.0, 0.0, 1e-3, 10)
    assert "Ricker" in api.sw_last_error()
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 2)(64, 64)
    spc = (ctypes.c_double * 2)(10.0, 10.0)
    faces = (ctypes.c_int * 4)(0, 0, 0, 0)
    # order 7 is rejected before any device work
    st = lib.sw_create_grid(ctypes.byref(h), 2, shp, spc, 7, faces, faces, 0.0, 3, 0.0, None)
    assert st == api.SW_EINVAL and h.value is None


def test_workloads_are_deterministic():
    a = workloads.make("3d_layered_256", shape=(40, 44, 48))
    b = workloads.make("3d_layered_256", shape=(40, 44, 48))
    assert np.array_equal(a.velocity, b.velocity)
    assert a.velocity.dtype == np.float32 and a.velocity.shape == (40, 44, 48)
    v = workloads.make("3d_vd_512x512x384", shape=(48, 40, 40))
    assert v.density is not None and v.order == 16
    c1 = workloads.make("2d_homogeneous_256")
    assert c1.updates == 256 * 256 * 1000 and len(c1.rec_pos) == 64


def test_binding_checks_buffer_sizes_before_the_call():
    """The C calls read and write whole buffers of the sizes the grid implies
    and cannot see the caller's: the binding refuses a buffer of the wrong size
    (and shot positions that do not match the acquisition's sources) before
    anything reaches the library.  A handle-less Grid stands in for a real one:
    every case must raise before the library is touched."""
    g = api.Grid(None, 3, (4, 5, 6), None)
    g.n_src, g.n_rec = 2, 7
    nodes = 4 * 5 * 6
    f32 = lambda n: np.zeros(n, np.float32)
    with pytest.raises(ValueError, match="velocity"):
        api.sw_set_model(g, f32(nodes - 1))
    with pytest.raises(ValueError, match="density"):
        api.sw_set_model(g, f32(nodes), f32(nodes + 1))
    with pytest.raises(ValueError, match="seismogram"):
        api.sw_forward(g, 10, f32(10 * 7 - 1))
    with pytest.raises(ValueError, match="final_field"):
        api.sw_forward(g, 10, f32(10 * 7), f32(nodes - 6))
    with pytest.raises(ValueError, match="observed"):
        api.sw_gradient(g, 10, f32(10 * 7 - 1), f32(nodes))
    with pytest.raises(ValueError, match="grad_vel"):
        api.sw_gradient(g, 10, f32(10 * 7), f32(nodes + 1))
    with pytest.raises(ValueError, match="grad_rho"):
        api.sw_gradient(g, 10, f32(10 * 7), f32(nodes), grad_rho=f32(1))
    # one position per shot while the acquisition has two sources
    with pytest.raises(ValueError, match="shot_src_pos"):
        api.sw_gradient_shots(g, np.zeros((3, 3)), 10, f32(3 * 10 * 7), f32(nodes))
    with pytest.raises(ValueError, match="observed"):
        api.sw_gradient_shots(g, np.zeros((3, 2, 3)), 10, f32(3 * 10 * 7 - 1), f32(nodes))
    with pytest.raises(ValueError, match="grad_vel"):
        api.sw_gradient_shots(g, np.zeros((3, 2, 3)), 10, f32(3 * 10 * 7), f32(nodes - 1))
    # one wavelet per source asked for, one wavelet given
    with pytest.raises(ValueError, match="wavelet"):
        api.sw_set_acquisition(g, np.zeros((2, 3)), np.zeros((7, 3)), f32(50), wavelet_per_source=True)


def test_binding_checks_batch_and_snapshot_buffers():
    """The same size checks for the snapshot frames and for a batch's per-grid
    outputs (one of each per grid, each of its own grid's size)."""
    g1 = api.Grid(None, 3, (4, 5, 6), None)
    g2 = api.Grid(None, 3, (3, 5, 6), None)
    g1.n_rec, g2.n_rec = 7, 2
    f32 = lambda n: np.zeros(n, np.float32)
    with pytest.raises(ValueError, match="snapshots"):
        api.sw_set_saving(g1, 5, f32(3 * 120 - 1), max_frames=3)
    b = api.Batch(None, [g1, g2])
    with pytest.raises(ValueError, match="per grid"):
        api.sw_batch_forward(b, 10, [f32(70)])
    with pytest.raises(ValueError, match="seismogram of grid 1"):
        api.sw_batch_forward(b, 10, [f32(70), f32(19)])
    with pytest.raises(ValueError, match="final field of grid 1"):
        api.sw_batch_forward(b, 10, [None, None], [f32(120), f32(120)])
