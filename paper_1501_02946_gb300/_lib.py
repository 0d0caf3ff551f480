"""ctypes declarations of the C ABI in include/pa_nufft.h.

Loading fails loudly: there is no CPU or library fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa_nufft.so")

PA_OK = 0
ERRORS = {1: "PA_ERR_INVALID_ARG", 2: "PA_ERR_UNSUPPORTED_SIZE", 3: "PA_ERR_CUDA", 4: "PA_ERR_OOM",
          5: "PA_ERR_TIMEOUT", 6: "PA_ERR_DEVICE"}


class PaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class PaGrid(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
                ("dx", c_double), ("dy", c_double), ("dz", c_double)]


class PaGrid2(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("nz", c_int32), ("dx", c_double), ("dz", c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "pa_plan_create": (c_int, [POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_int64, c_double, c_double,
                               POINTER(PaGrid), c_int, c_int, c_int, c_void_p]),
    "pa_plan_create_2d": (c_int, [POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_int64, c_double, c_double,
                                  POINTER(PaGrid2), c_int, c_int, c_int, c_void_p]),
    "pa_plan_dims": (c_int, [c_void_p, POINTER(c_int)]),
    "pa_correlation": (c_int, [c_void_p, c_void_p, c_int64, POINTER(c_double), c_void_p]),
    "pa_weight_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_voronoi_weights": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pa_plan_set_weights_device": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pa_voronoi_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_tenenbaum": (c_int, [c_void_p, c_int64, c_int64, c_int64, POINTER(c_double), c_void_p]),
    "pa_reconstruct": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_reconstruct_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_position_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_position_grad_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_plan_update_positions": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pa_plan_update_positions_device": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pa_plan_autotune": (c_int, [c_void_p, c_void_p, POINTER(c_int)]),
    "pa_plan_is_lattice": (c_int, [c_void_p, POINTER(c_int)]),
    "pa_plan_uses_warp_ner": (c_int, [c_void_p, POINTER(c_int)]),
    "pa_reconstruct_cubic": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pa_plan_destroy": (c_int, [c_void_p]),
    "pa_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p), c_void_p]),
    "pa_batch_run": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_void_p]),
    "pa_batch_destroy": (c_int, [c_void_p]),
    "pa_batch_set_mode": (c_int, [c_void_p, c_int]),
    "pa_status": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "pa_plan_test_wait_fault": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "pa_plan_info": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "pa_plan_buffer": (c_int, [c_void_p, c_int, c_void_p, c_int64, POINTER(c_int64), c_void_p]),
    "pa_profile_enable": (c_int, [c_void_p, c_int]),
    "pa_profile_select": (c_int, [c_void_p, ctypes.c_uint32]),
    "pa_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int64)]),
    "pa_profile_stage_name": (c_char_p, [c_int]),
    "pa_last_error": (c_char_p, []),
    "pa_version": (c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libpa_nufft.so (built in-tree by build.py) and declare signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1501_02946_gb300.build.build() "
                           "(the GPU path has no fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(rc):
    if rc != PA_OK:
        msg = load().pa_last_error()
        raise PaError(rc, msg.decode() if msg else "")
    return rc
