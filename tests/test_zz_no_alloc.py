"""accel_segreduce_noalloc: the segmented reduce for callers that cannot allocate device
memory (for example code running inside an allocator's hooks or under a host that owns
every allocation).  It uses a fixed scratch array built into the library instead of a
caller-provided workspace.  Its output must equal accel_segreduce's, bit for bit (integer
results), on two calls in a row sharing that array, and inputs beyond its limit must be
rejected without touching the GPU.

This file is collected last so that, if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2211_00621_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _case(seed, S, lo, hi):
    data, lengths = synth.ragged_flat_int32(seed, S, lo, hi)
    off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return torch.from_numpy(data).to(DEV), torch.from_numpy(off).to(DEV)


def _noalloc(lib, data, off, out):
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.accel_segreduce_noalloc(_lib.RED_ADD, _lib.MAP_SQ_PLUS_ONE, _lib.I32, _lib.I64,
                                       C.c_void_p(data.data_ptr()), data.numel(), C.c_void_p(off.data_ptr()),
                                       off.numel() - 1, 0.0, C.c_void_p(out.data_ptr()), st)


def test_noalloc_matches_workspace_entry_two_calls_in_a_row():
    lib = _lib.load()
    cases = [_case(0, 4096, 0, 256), _case(11, 50_000, 0, 300)]
    outs = []
    for data, off in cases:                       # two calls in a row share the scratch array
        out = torch.full((off.numel() - 1,), -7, dtype=torch.int64, device=DEV)
        _lib.check("accel_segreduce_noalloc", _noalloc(lib, data, off, out))
        outs.append(out)
    torch.cuda.synchronize()
    for (data, off), out in zip(cases, outs):
        ref = api.accel_segreduce(_lib.RED_ADD, _lib.MAP_SQ_PLUS_ONE, data, off, torch.int64)
        assert torch.equal(out, ref)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    lib = _lib.load()
    data, off = _case(1, 8, 0, 4)
    out = torch.empty(8, dtype=torch.int64, device=DEV)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.accel_segreduce_noalloc(_lib.RED_ADD, _lib.MAP_IDENTITY, _lib.I32, _lib.I64,
                                         C.c_void_p(data.data_ptr()), 178_913_281, C.c_void_p(off.data_ptr()),
                                         8, 0.0, C.c_void_p(out.data_ptr()), st)
    assert status == 7
    assert b"built-in area" in lib.accel_last_error()
