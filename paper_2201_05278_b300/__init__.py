"""B300-native (sm_103a) finite-difference acoustic wave solver.

Implements the explicit leapfrog solver of "simwave" (arXiv 2201.05278) as a
CUDA library with a C ABI (include/simwave_b300.h); this package is its thin
Python binding.  Importing it does not load the library; the first sw_* call
does, and raises if the library was not built.

    from paper_2201_05278_b300 import api
    g = api.sw_create_grid(3, (256, 256, 256), (10., 10., 10.), 8, nbl, bc, alpha, 3, dt)
    api.sw_set_model(g, velocity)                  # torch / numpy FP32, host or device
    api.sw_set_acquisition(g, src_pos, rec_pos, wavelet, window_radius=4)
    api.sw_forward(g, n_steps, seismogram, final_field)
"""
from . import api  # noqa: F401
from .api import (SimwaveError, sw_create_grid, sw_destroy_grid, sw_forward, sw_get_device_bytes,  # noqa: F401
                  sw_get_dt, sw_get_profile, sw_last_error, sw_ricker, sw_set_acquisition, sw_set_model,
                  sw_set_profiling)

__all__ = ["api", "SimwaveError", "sw_create_grid", "sw_destroy_grid", "sw_forward", "sw_get_device_bytes",
           "sw_get_dt", "sw_get_profile", "sw_last_error", "sw_ricker", "sw_set_acquisition", "sw_set_model",
           "sw_set_profiling"]
