"""ctypes declarations for libepcache (include/epcache.h)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
F32 = ctypes.c_float

# name -> (restype, argtypes); mirrors include/epcache.h
SIGNATURES = {
    "ep_version": (ctypes.c_int, []),
    "ep_last_error": (ctypes.c_char_p, []),
    "ep_partition": (ctypes.c_int, [P, P, I64, I64, I32, U32, I32, ctypes.POINTER(P)]),
    "ep_partition_start": (ctypes.c_int, [P, P, I64, I64, I32, U32, I32, ctypes.POINTER(P)]),
    "ep_job_wait": (ctypes.c_int, [P, I64, P]),
    "ep_job_take": (ctypes.c_int, [P, ctypes.POINTER(P), P]),
    "ep_job_cancel": (ctypes.c_int, [P]),
    "ep_job_free": (ctypes.c_int, [P]),
    "ep_schedule_info": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "ep_prescreen": (ctypes.c_int, [P, P, I64, I64, U32, P]),
    "ep_schedule_origin": (ctypes.c_int, [P, P]),
    "ep_schedule_arrays": (ctypes.c_int, [P, P, P, P, P, P]),
    "ep_cost_host": (ctypes.c_int, [P, P, P]),
    "ep_cost": (ctypes.c_int, [P, P, P, P]),
    "ep_run": (ctypes.c_int, [P, I32, P, P, P, I32, I32, F32, P]),
    "ep_run_host": (ctypes.c_int, [P, I32, P, P, P, I32, I32, F32, P]),
    "ep_run_adjoint": (ctypes.c_int, [P, P, P, P, P, I32, I32, F32, P]),
    "ep_record_floats": (I32, [I32]),
    "ep_layout_floats": (I64, [P, I32]),
    "ep_weights_floats": (I64, [P]),
    "ep_layout_in": (ctypes.c_int, [P, I32, P, P, P]),
    "ep_layout_out": (ctypes.c_int, [P, I32, P, P, P]),
    "ep_weights_in": (ctypes.c_int, [P, P, P, P]),
    "ep_weights_out_add": (ctypes.c_int, [P, P, P, P]),
    "ep_step": (ctypes.c_int, [P, I32, P, P, P, P, F32, P]),
    "ep_step_pending": (ctypes.c_int, [P, I32, P, P, P, F32, P]),
    "ep_finish": (ctypes.c_int, [P, I32, P, F32, P]),
    "ep_adjoint_step": (ctypes.c_int, [P, I32, P, P, P, P, F32, P]),
    "ep_adjoint_step_pending": (ctypes.c_int, [P, I32, P, P, P, P, F32, P]),
    "ep_adjoint_finish": (ctypes.c_int, [P, I32, P, F32, P]),
    "ep_spmv_x_in": (ctypes.c_int, [P, P, P, P]),
    "ep_spmv_y_out": (ctypes.c_int, [P, P, P, P]),
    "ep_spmv": (ctypes.c_int, [P, P, P, P, P]),
    "ep_batch": (ctypes.c_int, [P, I32, ctypes.POINTER(P)]),
    "ep_timing": (ctypes.c_int, [P, I32]),
    "ep_timing_read": (ctypes.c_int, [P, I32, P, P]),
    "ep_set_threads": (ctypes.c_int, [P, I32]),
    "ep_set_adjoint_threads": (ctypes.c_int, [P, I32]),
    "ep_set_halo": (ctypes.c_int, [P, P, I64]),
    "ep_halo_pack": (ctypes.c_int, [P, I32, P, P]),
    "ep_halo_unpack": (ctypes.c_int, [P, I32, P, P]),
    "ep_set_pipeline": (ctypes.c_int, [P, I32]),
    "ep_pipeline_info": (ctypes.c_int, [P, I32, I32, P, P, P, P, P]),
    "ep_check_errors": (ctypes.c_int, [P, P, P]),
    "ep_debug_stall": (ctypes.c_int, [P, I32]),
    "ep_set_cache": (ctypes.c_int, [P, I32]),
    "ep_schedule_free": (None, [P]),
    "ep_cost_noalloc": (ctypes.c_int, [P, P, P, I64, I64, I32, P, P]),
    "ep_noalloc_last_error": (ctypes.c_char_p, []),
}


class EpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libepcache error {code}: {msg}")
        self.code = code


def lib():
    """The loaded library (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libepcache.so is missing and could not be built")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(rc: int):
    if rc != 0:
        raise EpError(rc, lib().ep_last_error().decode(errors="replace"))
    return rc
