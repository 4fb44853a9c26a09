"""ctypes loader for libaccel.so and the C signatures of include/accel.h.

The library must exist (built by :func:`paper_2211_00621_gb300.build.build`); there is no
fallback: a missing or unloadable library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libaccel.so")

# status codes and constants (mirror include/accel.h)
ACCEL_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "DTYPE", 4: "WORKSPACE", 5: "CUDA",
                6: "TIMEOUT", 7: "UNSUPPORTED"}
I32, I64, F32, F64 = 0, 1, 2, 3
MAP_IDENTITY, MAP_SQ_PLUS_ONE, MAP_NEG, MAP_ABS, MAP_SCALE, MAP_ADD2, MAP_MUL2 = range(7)
RED_ADD, RED_MUL, RED_MIN, RED_MAX = range(4)
LOOP_AXPY, LOOP_SCALE = range(2)
PAIR_GRAVITY_SOFTENED = 0
HMM_FP32_LOG, HMM_BF16_SCALED = 0, 1
PROBE_FFMA, PROBE_FFMA2, PROBE_RSQRT, PROBE_DFMA = range(4)
MAX_RANK = 3


class AccelError(RuntimeError):
    def __init__(self, func: str, status: int, msg: str):
        self.status = status
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)} ({status}): {msg}")


class accel_tensor(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("rank", C.c_int32),
                ("dims", C.c_int64 * MAX_RANK)]


class accel_hmm_model(C.Structure):
    _fields_ = [("K", C.c_int32), ("M", C.c_int32), ("log_A", C.c_void_p), ("log_B", C.c_void_p),
                ("log_pi", C.c_void_p)]


vp, i32, i64, sz, dbl, flt = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double, C.c_float

# name -> (restype, argtypes)
SIGNATURES = {
    "accel_version": (C.c_char_p, []),
    "accel_last_error": (C.c_char_p, []),
    "accel_set_debug": (None, [i32]),
    "accel_get_debug": (i32, []),
    "accel_launch_count": (C.c_uint64, []),
    "accel_set_device_status": (i32, [vp]),
    "accel_sync_status": (i32, [vp, i32, vp]),
    "accel_set_watchdog_ns": (None, [C.c_uint64]),
    "accel_get_watchdog_ns": (C.c_uint64, []),
    "accel_set_sm_budget": (None, [C.c_int32]),
    "accel_get_sm_budget": (C.c_int32, []),
    "hmm_max_length": (i32, [vp, i64, vp, vp]),
    "accel_alu_rate": (i32, [i32, i64, vp, vp, vp]),
    "accel_marshal_ragged_workspace_size": (sz, [i64]),
    "accel_marshal_ragged": (i32, [vp, vp, i64, i32, vp, vp, vp, sz, vp]),
    "accel_marshal_nested_workspace_size": (sz, [i64, i64]),
    "accel_marshal_nested": (i32, [vp, vp, i64, vp, i64, i32, vp, vp, vp, vp, sz, vp]),
    "accel_unmarshal_ragged_workspace_size": (sz, [i64]),
    "accel_unmarshal_ragged": (i32, [vp, i64, vp, i64, i32, vp, vp, sz, vp]),
    "accel_marshal_records": (i32, [vp, i64, i32, i32, vp, vp, vp, i32, vp]),
    "accel_map": (i32, [i32, i32, vp, vp, i32, vp, i64, dbl, vp]),
    "accel_reduce_workspace_size": (sz, [i64, i32]),
    "accel_reduce": (i32, [i32, i32, vp, i64, vp, vp, sz, vp]),
    "accel_segreduce_workspace_size": (sz, [i64, i64]),
    "accel_segreduce": (i32, [i32, i32, i32, i32, vp, i64, vp, i64, dbl, vp, vp, sz, vp]),
    "accel_segreduce_noalloc": (i32, [i32, i32, i32, i32, vp, i64, vp, i64, dbl, vp, vp]),
    "accel_loop": (i32, [i32, i64, C.POINTER(accel_tensor), i32, dbl, vp]),
    "hmm_forward_workspace_size": (sz, [C.POINTER(accel_hmm_model), i64, i64, i32]),
    "hmm_forward": (i32, [C.POINTER(accel_hmm_model), i32, vp, vp, i64, i64, vp, vp, sz, vp]),
    "hmm_adjoint_workspace_size": (sz, [C.POINTER(accel_hmm_model), i64, i64, i64]),
    "hmm_adjoint": (i32, [C.POINTER(accel_hmm_model), vp, vp, i64, i64, i64, vp, vp, vp, vp, vp, vp, sz, vp]),
    "hmm_adjoint_forward": (i32, [C.POINTER(accel_hmm_model), vp, vp, i64, i64, i64, vp, vp, sz, vp]),
    "hmm_adjoint_backward": (i32, [C.POINTER(accel_hmm_model), vp, vp, i64, i64, i64, vp, vp, vp, vp, vp, sz, vp]),
    "pairwise_mapreduce": (i32, [i32, vp, vp, vp, vp, i64, flt, vp, vp, vp, vp]),
    "hmm_forward_long_workspace_size": (sz, [C.POINTER(accel_hmm_model), i64, i64, i64]),
    "hmm_forward_long": (i32, [C.POINTER(accel_hmm_model), vp, vp, i64, i64, i64, vp, vp, sz, vp]),
    "accel_pair_histogram": (i32, [vp, vp, vp, i64, vp, vp, vp, i64, vp, i32, vp, vp]),
    "hmm_mstep": (i32, [C.POINTER(accel_hmm_model), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "hmm_autotune": (i32, [C.POINTER(accel_hmm_model), i32, vp, vp, i64, i64, vp, vp, sz, C.c_char_p, vp, vp]),
    "hmm_tuned_config": (i32, [i32, i32, i64, vp, vp, vp, vp]),
    "accel_graph_begin": (i32, [vp]),
    "accel_graph_end": (i32, [vp, vp]),
    "accel_graph_launch": (i32, [vp, vp]),
    "accel_graph_destroy": (i32, [vp]),
    "accel_graph_node_count": (i32, [vp, vp]),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libaccel.so and declare its signatures (once)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"libaccel.so not found at {path}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (the CUDA library is required, "
                "there is no CPU fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(func: str, status: int):
    if status != ACCEL_OK:
        msg = load().accel_last_error().decode(errors="replace")
        raise AccelError(func, status, msg)
