"""Two-level flatten ([[[T]]]) and the device-to-host unmarshal of ragged results, against
the oracle, through the C ABI (bit-exact)."""
import numpy as np
import pytest
import torch

from oracle import patterns as op
from paper_2211_00621_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _groups(seed, G, max_seqs=5, max_len=40, dtype=np.int32):
    g = synth.rng(seed)
    out = []
    for _ in range(G):
        n = int(g.integers(0, max_seqs + 1))
        out.append([g.integers(-1000, 1000, size=int(g.integers(0, max_len + 1))).astype(dtype) for _ in range(n)])
    return out


def _to(groups, pinned):
    if pinned:
        return [[torch.from_numpy(s).pin_memory() for s in g] for g in groups]
    return [[torch.from_numpy(s).to(DEV) for s in g] for g in groups]


@pytest.mark.parametrize("pinned", [False, True])
def test_marshal_nested_matches_oracle(pinned):
    groups = _groups(1, 300)
    groups[0] = []                                          # an empty group first
    flat, off, goff = api.accel_marshal_nested(_to(groups, pinned))
    rf, ro, rg = op.marshal_nested(groups)
    assert np.array_equal(flat.cpu().numpy(), rf)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(goff.cpu().numpy(), rg)


def test_marshal_nested_int64_and_degenerate_shapes():
    groups = _groups(2, 50, dtype=np.int64)
    flat, off, goff = api.accel_marshal_nested(_to(groups, False), dtype=torch.int64)
    rf, ro, rg = op.marshal_nested(groups)
    assert np.array_equal(flat.cpu().numpy(), rf) and np.array_equal(goff.cpu().numpy(), rg)
    # no groups; groups holding only empty sequences
    flat, off, goff = api.accel_marshal_nested([])
    assert flat.numel() == 0 and off.cpu().tolist() == [0] and goff.cpu().tolist() == [0]
    z = [[np.zeros(0, np.int32)] * 3, []]
    flat, off, goff = api.accel_marshal_nested(_to(z, False))
    assert flat.numel() == 0 and off.cpu().tolist() == [0, 0, 0, 0] and goff.cpu().tolist() == [0, 3, 3]


def test_nested_reduce_of_reduces():
    # map (lam g. reduce (+) 0 (map (lam s. reduce (+) 0 (map (x*x+1) s)) g)): two segmented reduces
    groups = _groups(3, 2000, max_seqs=8, max_len=100)
    flat, off, goff = api.accel_marshal_nested(_to(groups, False))
    inner = api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, flat, off, torch.int64)
    outer = api.accel_segreduce(api.RED_ADD, api.MAP_IDENTITY, inner, goff, torch.int64)
    rf, ro, rg = op.marshal_nested(groups)
    r_in = op.segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, rf, ro, np.int64)
    r_out = op.segreduce(op.RED_ADD, op.MAP_IDENTITY, r_in, rg, np.int64)
    assert np.array_equal(outer.cpu().numpy(), r_out)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_unmarshal_ragged_roundtrip(pinned, dtype):
    seqs = synth.ragged_int32(7, 3000, 0, 300)
    seqs = [s.astype(dtype) for s in seqs]
    seqs[5] = seqs[5][:0]
    flat, off = api.accel_marshal_ragged([torch.from_numpy(s).to(DEV) for s in seqs],
                                         dtype=torch.int32 if dtype == np.int32 else torch.int64)
    back = api.accel_unmarshal_ragged(flat, off, pinned=pinned)
    ref = op.unmarshal_ragged(*op.marshal_ragged(seqs))
    assert len(back) == len(ref)
    for b, r in zip(back, ref):
        assert b.numel() == 0 or (b.is_pinned() if pinned else b.is_cuda)
        assert np.array_equal(b.cpu().numpy(), r)


def test_unmarshal_ragged_of_a_result():
    # results converted back: per-sequence x*x+1 (map over the flat data), unmarshaled
    seqs = synth.ragged_int32(8, 700, 0, 64)
    flat, off = api.accel_marshal_ragged([torch.from_numpy(s).to(DEV) for s in seqs])
    mapped = api.accel_map(api.MAP_SQ_PLUS_ONE, flat, torch.int64)
    back = api.accel_unmarshal_ragged(mapped, off)
    for b, s in zip(back, seqs):
        assert np.array_equal(b.numpy(), op.map_op(op.MAP_SQ_PLUS_ONE, s, np.int64))
    assert api.accel_unmarshal_ragged(flat[:0], torch.zeros(1, dtype=torch.int64, device=DEV)) == []
