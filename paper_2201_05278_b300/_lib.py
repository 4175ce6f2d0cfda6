"""ctypes loader for the in-tree CUDA library libsimwave_b300.so.

There is no fallback: if the library is missing or cannot be loaded, every
call raises.  The symbols and their C signatures are those of
include/simwave_b300.h.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsimwave_b300.so")

# name -> (restype, argtypes), mirroring include/simwave_b300.h
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_dp = ctypes.POINTER(ctypes.c_double)
_c_ip = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "sw_create_grid": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_i64p, _c_dp,
                                      ctypes.c_int, _c_ip, _c_ip, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p]),
    "sw_set_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sw_set_acquisition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dp, ctypes.c_int, _c_dp,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sw_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "sw_get_dt": (ctypes.c_int, [ctypes.c_void_p, _c_dp]),
    "sw_ricker": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_void_p]),
    "sw_set_stencil_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sw_set_pipeline_test": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_ulonglong]),
    "sw_set_saving": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]),
    "sw_set_checkpoint_budget": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sw_set_forcing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "sw_set_initial_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sw_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sw_gradient_shots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dp, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_int]),
    "sw_get_stencil_variant": (ctypes.c_int, [ctypes.c_void_p, _c_ip]),
    "sw_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sw_get_profile": (ctypes.c_int, [ctypes.c_void_p, _c_dp, _c_i64p, _c_i64p]),
    "sw_get_device_bytes": (ctypes.c_int, [ctypes.c_void_p, _c_i64p]),
    "sw_forward_noalloc": (ctypes.c_int, [ctypes.c_int, _c_i64p, _c_dp, ctypes.c_int, _c_ip, _c_ip,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, _c_dp, ctypes.c_int, _c_dp, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sw_last_error": (ctypes.c_char_p, []),
    "sw_destroy_grid": (None, [ctypes.c_void_p]),
    "sw_create_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.c_int]),
    "sw_batch_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "sw_batch_info": (ctypes.c_int, [ctypes.c_void_p, _c_ip, _c_ip]),
    "sw_batch_get_tile": (ctypes.c_int, [ctypes.c_void_p, _c_ip, ctypes.POINTER(ctypes.c_float)]),
    "sw_batch_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sw_batch_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sw_batch_get_profile": (ctypes.c_int, [ctypes.c_void_p, _c_dp, _c_i64p, _c_i64p]),
    "sw_destroy_batch": (None, [ctypes.c_void_p]),
}

_lib = None


def load():
    """Load libsimwave_b300.so (raises OSError if it is absent or broken)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libsimwave_b300.so not built: run __graft_entry__.build() "
                          "or python paper_2201_05278_b300/build.py")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
