"""accel_segreduce_noalloc: the segmented reduce for callers that cannot allocate device
memory (for example code running inside an allocator's hooks or under a host that owns
every allocation).  It uses a fixed scratch array built into the library instead of a
caller-provided workspace.  Its output must equal accel_segreduce's on two calls in a row
sharing that array (bit for bit for integer results, within the summation bound for float
sums), on every kernel path of the shared implementation (the integer prefix-sum path, the
general fold for other operators and for floats), up to and including its size limit, and
inputs beyond that limit must be rejected without touching the GPU.

This file is collected last so that, if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2211_00621_gb300 import _lib, api, synth
from oracle import patterns as op

pytestmark = pytest.mark.gpu
DEV = "cuda"
LIMIT = 178_913_280          # the largest N the built-in scratch array serves

_NP = {_lib.I32: np.int32, _lib.I64: np.int64, _lib.F32: np.float32, _lib.F64: np.float64}
_TORCH = {_lib.I32: torch.int32, _lib.I64: torch.int64, _lib.F32: torch.float32, _lib.F64: torch.float64}


def _case(seed, S, lo, hi, in_dt=_lib.I32):
    data, lengths = synth.ragged_flat_int32(seed, S, lo, hi)
    if in_dt == _lib.F32:
        data = (data.astype(np.float64) / 7.0).astype(np.float32)
    off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return data, off


def _noalloc(lib, red, fmap, in_dt, out_dt, data, off, out, scalar=0.0):
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.accel_segreduce_noalloc(red, fmap, in_dt, out_dt, C.c_void_p(data.data_ptr()), data.numel(),
                                       C.c_void_p(off.data_ptr()), off.numel() - 1, scalar,
                                       C.c_void_p(out.data_ptr()), st)


# (reduce, fused map, input type, output type): the integer sum of x*x+1 runs the prefix-sum
# kernel; MAX over int32 and the float32 sum run the general fold with its carry fix-up
PATHS = [(_lib.RED_ADD, _lib.MAP_SQ_PLUS_ONE, _lib.I32, _lib.I64),
         (_lib.RED_MAX, _lib.MAP_IDENTITY, _lib.I32, _lib.I32),
         (_lib.RED_ADD, _lib.MAP_IDENTITY, _lib.F32, _lib.F32)]


def _check(red, fmap, in_dt, out_dt, data, off, got):
    ref_ws = api.accel_segreduce(red, fmap, torch.from_numpy(data).to(DEV), torch.from_numpy(off).to(DEV),
                                 _TORCH[out_dt]).cpu().numpy()
    ref = op.segreduce(red, fmap, data, off, _NP[out_dt])
    if np.dtype(_NP[out_dt]).kind == "i":
        assert np.array_equal(got, ref_ws)
        assert np.array_equal(got, ref)
    else:
        # float sums: the same order as the workspace entry point, and within n u sum|x| of
        # the float64 oracle
        assert np.array_equal(got, ref_ws)
        u = np.finfo(np.float32).eps / 2
        n = np.maximum(np.diff(off), 1)
        absum = op.segreduce(op.RED_ADD, op.MAP_ABS, data, off, np.float64)
        assert np.all(np.abs(got.astype(np.float64) - ref) <= 2 * n * u * absum + 1e-30)


@pytest.mark.parametrize("red,fmap,in_dt,out_dt", PATHS)
def test_noalloc_matches_workspace_entry_two_calls_in_a_row(red, fmap, in_dt, out_dt):
    lib = _lib.load()
    cases = [_case(0, 4096, 0, 256, in_dt), _case(11, 20_000, 0, 300, in_dt)]
    outs = []
    for data, off in cases:                       # two calls in a row share the scratch array
        out = torch.full((len(off) - 1,), -7, dtype=_TORCH[out_dt], device=DEV)
        _lib.check("accel_segreduce_noalloc", _noalloc(lib, red, fmap, in_dt, out_dt, torch.from_numpy(data).to(DEV),
                                                       torch.from_numpy(off).to(DEV), out))
        outs.append(out)
    torch.cuda.synchronize()
    for (data, off), out in zip(cases, outs):
        _check(red, fmap, in_dt, out_dt, data, off, out.cpu().numpy())


def test_noalloc_at_its_size_limit():
    # N exactly at the limit: 698,880 segments of 256 int32 elements (the most tiles the
    # array holds), then a small call right after it in the same array
    lib = _lib.load()
    S = LIMIT // 256
    g = synth.rng(17)
    data = g.integers(-1000, 1001, size=LIMIT, dtype=np.int64).astype(np.int32)
    off = np.arange(S + 1, dtype=np.int64) * 256
    d_data, d_off = torch.from_numpy(data).to(DEV), torch.from_numpy(off).to(DEV)
    out = torch.empty(S, dtype=torch.int64, device=DEV)
    _lib.check("accel_segreduce_noalloc", _noalloc(lib, _lib.RED_ADD, _lib.MAP_SQ_PLUS_ONE, _lib.I32, _lib.I64,
                                                   d_data, d_off, out))
    small_data, small_off = _case(3, 1000, 0, 64)
    small_out = torch.empty(1000, dtype=torch.int64, device=DEV)
    _lib.check("accel_segreduce_noalloc", _noalloc(lib, _lib.RED_ADD, _lib.MAP_SQ_PLUS_ONE, _lib.I32, _lib.I64,
                                                   torch.from_numpy(small_data).to(DEV),
                                                   torch.from_numpy(small_off).to(DEV), small_out))
    ref = op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, np.int64)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(small_out.cpu().numpy(),
                          op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, small_data, small_off, np.int64))


def test_noalloc_rejects_inputs_beyond_its_scratch():
    lib = _lib.load()
    data, off = _case(1, 8, 0, 4)
    out = torch.empty(8, dtype=torch.int64, device=DEV)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    d_data, d_off = torch.from_numpy(data).to(DEV), torch.from_numpy(off).to(DEV)
    status = lib.accel_segreduce_noalloc(_lib.RED_ADD, _lib.MAP_IDENTITY, _lib.I32, _lib.I64,
                                         C.c_void_p(d_data.data_ptr()), LIMIT + 1, C.c_void_p(d_off.data_ptr()),
                                         8, 0.0, C.c_void_p(out.data_ptr()), st)
    assert status == 7
    assert b"built-in area" in lib.accel_last_error()
    # an error found by the shared implementation names this entry point
    status = lib.accel_segreduce_noalloc(_lib.RED_ADD, _lib.MAP_IDENTITY, _lib.I32, _lib.F32,
                                         C.c_void_p(d_data.data_ptr()), d_data.numel(),
                                         C.c_void_p(d_off.data_ptr()), 8, 0.0, C.c_void_p(out.data_ptr()), st)
    assert status != 0
    assert lib.accel_last_error().startswith(b"accel_segreduce_noalloc")
