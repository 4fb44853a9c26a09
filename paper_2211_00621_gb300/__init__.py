"""GB300 (sm_103a) library for the data-parallel hot path of expression acceleration
(Expression Acceleration: Seamless Parallelization of Typed High-Level Languages,
arXiv 2211.00621): marshaling of ragged sequences and records, map / map2 / reduce /
segmented reduce / loop over a fixed operator set, the HMM forward recursion (FP32
log-space and BF16 tensor-core scaled forms) with its adjoint, and an all-pairs
map-of-reduce.

The compute path is the C-ABI library ``libaccel.so`` (hand-written CUDA, see
``include/accel.h``); :mod:`.api` is its PyTorch binding.  Importing this package does
not load the library; the first call does, and fails if it is missing.
"""
from ._lib import (  # noqa: F401
    AccelError, HMM_BF16_SCALED, HMM_FP32_LOG, I32, I64, F32, F64, LOOP_AXPY, LOOP_SCALE, MAP_ABS, MAP_ADD2,
    MAP_IDENTITY, MAP_MUL2, MAP_NEG, MAP_SCALE, MAP_SQ_PLUS_ONE, PAIR_GRAVITY_SOFTENED, RED_ADD, RED_MAX,
    RED_MIN, RED_MUL,
)


_API = {"accel_marshal_ragged", "accel_marshal_ragged_table", "accel_marshal_nested", "accel_unmarshal_ragged", "ragged_table", "accel_marshal_records", "accel_map", "accel_reduce", "accel_segreduce",
        "accel_loop", "hmm_forward", "hmm_forward_long", "hmm_adjoint", "hmm_mstep", "hmm_autotune", "Graph", "HMMLogLik", "pairwise_mapreduce", "accel_pair_histogram",
        "set_debug", "version", "set_device_status", "sync_status", "set_watchdog_ns", "set_sm_budget", "get_sm_budget", "hmm_max_length", "alu_rate",
        "hmm_adjoint_forward", "hmm_adjoint_backward"}


def __getattr__(name):
    # lazy: the binding imports torch
    if name in _API:
        import importlib
        return getattr(importlib.import_module(__name__ + ".api"), name)
    raise AttributeError(name)
