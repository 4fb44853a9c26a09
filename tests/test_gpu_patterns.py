"""GPU parity of the pattern kernels (marshal, map, reduce, segmented reduce, loop) with
the CPU oracle, through the C ABI.  Integer results must be bit-exact."""
import math

import numpy as np
import pytest
import torch

import paper_2211_00621_gb300 as acc
from paper_2211_00621_gb300 import api, synth
from oracle import patterns as op

pytestmark = pytest.mark.gpu
DEV = "cuda"

TORCH_DT = {np.int32: torch.int32, np.int64: torch.int64, np.float32: torch.float32, np.float64: torch.float64}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# ----------------------------------------------------------------------------- marshal
def test_marshal_ragged_device_pieces_config():
    c = synth.CFG_SEGREDUCE
    seqs = synth.ragged_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
    flat, off = api.accel_marshal_ragged([_t(s) for s in seqs])
    rf, ro = op.marshal_ragged(seqs)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(flat.cpu().numpy(), rf)


def test_marshal_ragged_pinned_host_pieces_and_empties():
    seqs = synth.ragged_int32(3, 500, 0, 40)
    seqs[0] = seqs[0][:0]
    seqs[-1] = seqs[-1][:0]
    pieces = [torch.from_numpy(s).pin_memory() for s in seqs]
    flat, off = api.accel_marshal_ragged(pieces)
    rf, ro = op.marshal_ragged(seqs)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(flat.cpu().numpy(), rf)


def test_marshal_ragged_int64_and_many_sequences():
    g = synth.rng(9)
    seqs = [g.integers(-2**40, 2**40, size=int(n), dtype=np.int64) for n in g.integers(0, 5, size=5000)]
    flat, off = api.accel_marshal_ragged([_t(s) for s in seqs], dtype=torch.int64)
    rf, ro = op.marshal_ragged(seqs)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(flat.cpu().numpy(), rf)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("S", [16 * 1024, 16 * 1024 + 1, 40_000, 200_003])
def test_marshal_ragged_scan_paths(S, pinned):
    # S <= 16,384 scans the lengths in one CTA, larger S in three passes (200,003: more
    # sequences per warp batch, a partial last batch); page-locked host tables are read in
    # place by the kernels, pageable ones are copied to the workspace first
    seqs = synth.ragged_int32(S, S, 0, 9)
    pieces = [_t(x) for x in seqs]
    ptrs = torch.tensor([p.data_ptr() if p.numel() else 0 for p in pieces], dtype=torch.int64)
    lens = torch.tensor([p.numel() for p in pieces], dtype=torch.int64)
    if pinned:
        ptrs, lens = ptrs.pin_memory(), lens.pin_memory()
    lib = api.L.load()
    total = int(lens.sum())
    flat = torch.empty(total, dtype=torch.int32, device=DEV)
    off = torch.empty(S + 1, dtype=torch.int64, device=DEV)
    ws = torch.empty(lib.accel_marshal_ragged_workspace_size(S), dtype=torch.uint8, device=DEV)
    import ctypes as C
    api.L.check("accel_marshal_ragged", lib.accel_marshal_ragged(
        C.c_void_p(ptrs.data_ptr()), C.c_void_p(lens.data_ptr()), S, api.L.I32, C.c_void_p(flat.data_ptr()),
        C.c_void_p(off.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
        C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    rf, ro = op.marshal_ragged(seqs)
    assert np.array_equal(off.cpu().numpy(), ro)
    assert np.array_equal(flat.cpu().numpy(), rf)


def test_marshal_ragged_sweep_size_shuffled_pieces():
    # 2^20 sequences (lengths U{0..256}, ~134M elements) whose pieces lie in one buffer in a
    # shuffled order: the HBM-scale marshal the bench times, compared element by element
    S = 1 << 20
    data, lengths = synth.ragged_flat_int32(1, S)
    perm = synth.rng(5).permutation(S)
    start = np.zeros(S, np.int64)
    start[perm] = np.concatenate([[0], np.cumsum(lengths[perm])[:-1]])
    src = np.empty_like(data)
    ref_off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=ref_off[1:])
    for_src = np.repeat(start - ref_off[:-1], lengths) + np.arange(len(data))   # source position of flat k
    src[for_src] = data
    d_src = _t(src)
    table = api.RaggedTable.__new__(api.RaggedTable)
    table.seqs, table.dtype, table.S = [d_src], torch.int32, S
    tab = torch.from_numpy(np.concatenate([d_src.data_ptr() + 4 * start, lengths]).astype(np.int64)).pin_memory()
    table.ptrs, table.lengths, table.total = tab[:S], tab[S:], int(lengths.sum())
    flat, off = api.accel_marshal_ragged_table(table)
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy(), ref_off)
    assert np.array_equal(flat.cpu().numpy(), data)


def test_seg_row_captured_as_one_graph_replays():
    # marshal -> fused map + segmented sum -> max -> loop, captured once and replayed twice
    c = synth.CFG_SEGREDUCE
    seqs = synth.ragged_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
    table = api.ragged_table([_t(x) for x in seqs])
    lib = api.L.load()
    N, S = table.total, table.S
    flat = torch.empty(N, dtype=torch.int32, device=DEV)
    off = torch.empty(S + 1, dtype=torch.int64, device=DEV)
    seg = torch.empty(S, dtype=torch.int64, device=DEV)
    mx = torch.empty(1, dtype=torch.int64, device=DEV)
    twice = torch.empty(N, dtype=torch.int32, device=DEV)
    ws_m = torch.empty(lib.accel_marshal_ragged_workspace_size(S), dtype=torch.uint8, device=DEV)
    ws_s = torch.empty(lib.accel_segreduce_workspace_size(N, S), dtype=torch.uint8, device=DEV)
    ws_r = torch.empty(max(lib.accel_reduce_workspace_size(S, api.L.I64), 256), dtype=torch.uint8, device=DEV)

    def body():
        api.accel_marshal_ragged_table(table, out=(flat, off), ws=ws_m)
        api.accel_segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, flat, off, torch.int64, out=seg, ws=ws_s)
        api.accel_reduce(op.RED_MAX, seg, out=mx, ws=ws_r)
        api.accel_loop(op.LOOP_SCALE, twice, flat, 2.0)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = api.Graph()
    g.capture(body, stream=side)
    rf, ro = op.marshal_ragged(seqs)
    ref = op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, rf, ro, np.int64)
    for _ in range(2):
        for t in (flat, seg, mx, twice):
            t.fill_(-1)
        torch.cuda.synchronize()
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(seg.cpu().numpy(), ref)
        assert int(mx.item()) == int(ref.max())
        assert np.array_equal(twice.cpu().numpy(), 2 * rf)


def test_marshal_records_fast_path_and_inverse():
    b = synth.bodies(2, 1001)
    aos = _t(b["aos"])
    f32 = torch.float32
    cols = api.accel_marshal_records(aos, [(0, f32), (4, f32), (8, f32), (12, f32)])
    ref = op.marshal_records(b["aos"].view(np.uint8).reshape(1001, 16),
                             [(0, np.float32), (4, np.float32), (8, np.float32), (12, np.float32)])
    for c, r in zip(cols, ref):
        assert np.array_equal(c.cpu().numpy(), r)
    back = torch.zeros_like(aos)
    api.accel_marshal_records(back, [(0, f32), (4, f32), (8, f32), (12, f32)], inverse_from=cols)
    assert torch.equal(back, aos)


def test_marshal_records_general_layout():
    # record {a: int32 @0, b: float64 @8, c: float32 @16, pad} of 24 bytes
    n = 777
    g = synth.rng(4)
    raw = g.integers(0, 256, size=(n, 24), dtype=np.int64).astype(np.uint8)
    fields = [(0, np.int32), (8, np.float64), (16, np.float32)]
    ref = op.marshal_records(raw, fields)
    aos = _t(raw)
    cols = api.accel_marshal_records(aos, [(o, TORCH_DT[d]) for o, d in fields])
    for c, r in zip(cols, ref):
        assert np.array_equal(c.cpu().numpy().view(np.uint8), r.view(np.uint8))
    back = torch.zeros_like(aos)
    api.accel_marshal_records(back, [(o, TORCH_DT[d]) for o, d in fields], inverse_from=cols)
    refb = op.unmarshal_records(ref, fields, 24)
    assert np.array_equal(back.cpu().numpy(), refb)


# --------------------------------------------------------------------------------- map
@pytest.mark.parametrize("op_id", [op.MAP_IDENTITY, op.MAP_SQ_PLUS_ONE, op.MAP_NEG, op.MAP_ABS, op.MAP_SCALE,
                                   op.MAP_ADD2, op.MAP_MUL2])
@pytest.mark.parametrize("dts", [(np.int32, np.int64), (np.int32, np.int32), (np.int64, np.int64),
                                 (np.float32, np.float32), (np.float64, np.float64), (np.int32, np.float64)])
def test_map_ops(op_id, dts):
    din, dout = dts
    n = 1000 + 37
    g = synth.rng(op_id * 7 + 1)
    if np.dtype(din).kind == "i":
        x = g.integers(-100000, 100000, size=n).astype(din)
        y = g.integers(-100000, 100000, size=n).astype(din)
    else:
        x = g.standard_normal(n).astype(din)
        y = g.standard_normal(n).astype(din)
    binary = op_id in (op.MAP_ADD2, op.MAP_MUL2)
    out = api.accel_map(op_id, _t(x), TORCH_DT[dout], _t(y) if binary else None, scalar=3.0)
    ref = op.map_op(op_id, x, dout, y if binary else None, scalar=3.0)
    got = out.cpu().numpy()
    if np.dtype(dout).kind == "i":
        assert np.array_equal(got, ref)
    else:
        tol = 2e-6 if dout == np.float32 else 1e-14
        np.testing.assert_allclose(got, ref, rtol=tol, atol=tol)


def test_map_unaligned_and_empty():
    x = np.arange(-50, 51, dtype=np.int32)
    tx = _t(np.concatenate([[7], x]))[1:]          # 4-byte offset: not 16-byte aligned
    out = api.accel_map(op.MAP_SQ_PLUS_ONE, tx, torch.int64)
    assert np.array_equal(out.cpu().numpy(), x.astype(np.int64) ** 2 + 1)
    e = api.accel_map(op.MAP_NEG, _t(np.zeros(0, np.int32)))
    assert e.numel() == 0


# ------------------------------------------------------------------------------ reduce
# n <= 65,536 is reduced by one CTA, larger n in two passes
@pytest.mark.parametrize("n", [200_003, 65_537, 65_536, 4_097, 1])
@pytest.mark.parametrize("red", [op.RED_ADD, op.RED_MUL, op.RED_MIN, op.RED_MAX])
@pytest.mark.parametrize("dt", [np.int32, np.int64])
def test_reduce_int_bit_exact(red, dt, n):
    g = synth.rng(red + 11)
    x = g.integers(-5 if red == op.RED_MUL else -10**6, 6 if red == op.RED_MUL else 10**6, size=n).astype(dt)
    got = api.accel_reduce(red, _t(x)).item()
    if red == op.RED_MUL:
        m = min(n, 2000)
        ref = op.reduce_op(red, x[:m])             # wrapping product: compare a prefix exactly
        got = api.accel_reduce(red, _t(x[:m])).item()
    elif red == op.RED_ADD:
        ref = int(np.sum(x.astype(np.int64)))
        bits = np.dtype(dt).itemsize * 8
        ref = ((ref + (1 << (bits - 1))) % (1 << bits)) - (1 << (bits - 1))
    elif red == op.RED_MIN:
        ref = int(x.min())
    else:
        ref = int(x.max())
    assert got == ref


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_reduce_float(dt):
    n = 1_000_001
    x = synth.rng(5).standard_normal(n).astype(dt)
    got = api.accel_reduce(op.RED_ADD, _t(x)).item()
    ref = math.fsum(x.astype(np.float64).tolist())
    bound = n * (2.0 ** -24 if dt == np.float32 else 2.0 ** -53) * float(np.abs(x).sum())
    assert abs(got - ref) <= bound
    assert api.accel_reduce(op.RED_MAX, _t(x)).item() == float(x.max())


@pytest.mark.parametrize("dt", [np.int64, np.int32])
def test_reduce_empty_gives_neutral(dt):
    # the neutral element of the result's own type (an int32 reduction runs in int64, but an
    # empty one gives INT32_MIN / INT32_MAX, not a narrowed int64 value)
    e = _t(np.zeros(0, dt))
    for red in (op.RED_ADD, op.RED_MUL, op.RED_MIN, op.RED_MAX):
        assert api.accel_reduce(red, e).item() == op.neutral(red, dt)
    assert op.neutral(op.RED_MAX, dt) == np.iinfo(dt).min


# ----------------------------------------------------------------------- segreduce
def _seg_case(seed, S, lo, hi, dt=np.int32):
    g = synth.rng(seed)
    lengths = g.integers(lo, hi + 1, size=S)
    total = int(lengths.sum())
    if np.dtype(dt).kind == "i":
        data = g.integers(-1000, 1001, size=total).astype(dt)
    else:
        data = g.standard_normal(total).astype(dt)
    off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return data, off


def test_segreduce_config_bit_exact_and_max():
    c = synth.CFG_SEGREDUCE
    seqs = synth.ragged_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
    flat, off = api.accel_marshal_ragged([_t(s) for s in seqs])
    seg = api.accel_segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, flat, off, torch.int64)
    mx = api.accel_reduce(op.RED_MAX, seg)
    rf, ro = op.marshal_ragged(seqs)
    ref = op.segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, rf, ro, np.int64)
    assert np.array_equal(seg.cpu().numpy(), ref)
    assert mx.item() == int(ref.max())
    # sum of segment sums equals the total (fixed by associativity)
    assert int(seg.sum().item()) == int(np.sum(rf.astype(np.int64) ** 2 + 1))


# Inputs of at most 2^20 elements (segments of at most 4,096 elements on average) take the
# one-warp-per-segment kernel; larger ones the tiled kernels.  PATH "tiled" appends a segment
# of 2^20 + 1 zeros after the case, which sends the same segments through the tiled kernels;
# the appended segment's result is checked on its own.
PATHS = ["warp", "tiled"]
TAIL = (1 << 20) + 1


def _with_tail(data, off, path):
    if path == "warp":
        return data, off
    data2 = np.concatenate([data, np.zeros(TAIL, data.dtype)])
    off2 = np.concatenate([off, [off[-1] + TAIL]]).astype(np.int64)
    return data2, off2


def _tail_value(red, fmap, scalar=0.0):
    g0 = {op.MAP_IDENTITY: 0, op.MAP_SQ_PLUS_ONE: 1, op.MAP_NEG: 0, op.MAP_ABS: 0, op.MAP_SCALE: 0}[fmap]
    return {op.RED_ADD: g0 * TAIL, op.RED_MUL: g0, op.RED_MIN: g0, op.RED_MAX: g0}[red]


def _segreduce_path(red, fmap, data, off, dt, path, scalar=0.0):
    d2, o2 = _with_tail(data, off, path)
    got = api.accel_segreduce(red, fmap, _t(d2), _t(o2), dt, scalar=scalar).cpu().numpy()
    if path == "tiled":
        assert got[-1] == _tail_value(red, fmap, scalar)
        got = got[:-1]
    return got


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("red", [op.RED_ADD, op.RED_MUL, op.RED_MIN, op.RED_MAX])
@pytest.mark.parametrize("fmap", [op.MAP_IDENTITY, op.MAP_SQ_PLUS_ONE, op.MAP_NEG, op.MAP_ABS, op.MAP_SCALE])
def test_segreduce_ops_small(red, fmap, path):
    data, off = _seg_case(red * 10 + fmap, 300, 0, 60)
    if red == op.RED_MUL:
        data = (data % 5).astype(np.int32)
    got = _segreduce_path(red, fmap, data, off, torch.int64, path, scalar=-2.0)
    ref = op.segreduce(red, fmap, data, off, np.int64, scalar=-2.0)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("case", ["one_long", "all_empty_tail", "unit_lengths", "empty_runs", "spanning_tiles"])
def test_segreduce_edge_cases(case, path):
    g = synth.rng(1)
    if case == "one_long":            # one segment spanning many tiles
        lengths = np.array([100_003])
    elif case == "all_empty_tail":    # non-empty then empties positioned at N
        lengths = np.array([5000, 4096, 0, 0, 0])
    elif case == "unit_lengths":      # > 1024 segments per tile: offsets not cached in shared memory
        lengths = g.integers(0, 2, size=40_000)
    elif case == "empty_runs":        # empties at tile and thread boundaries
        lengths = np.array([16, 0, 0, 4080, 0, 16, 0, 0, 4096, 0, 1, 0] * 50)
    else:                             # segments of ~3 tiles interleaved with short ones
        lengths = np.tile([12_000, 3, 0, 7], 20)
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    data = g.integers(-1000, 1001, size=int(off[-1])).astype(np.int32)
    for red in (op.RED_ADD, op.RED_MAX):
        got = _segreduce_path(red, op.MAP_SQ_PLUS_ONE, data, off, torch.int64, path)
        ref = op.segreduce_fast(red, op.MAP_SQ_PLUS_ONE, data, off, np.int64)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("dout", [np.int64, np.int32])
def test_segreduce_no_elements(dout):
    off = np.zeros(17, np.int64)
    for red in (op.RED_MIN, op.RED_MAX, op.RED_MUL):
        got = api.accel_segreduce(red, op.MAP_IDENTITY, _t(np.zeros(0, np.int32)), _t(off), TORCH_DT[dout])
        assert np.array_equal(got.cpu().numpy(), np.full(16, op.neutral(red, dout), dtype=dout))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("red", [op.RED_MIN, op.RED_MAX, op.RED_ADD])
def test_segreduce_int32_output_with_empty_segments(red, path):
    # an empty segment gives the int32 neutral element, at every position in a tile
    data, off = _seg_case(40 + red, 3000, 0, 12)
    got = _segreduce_path(red, op.MAP_IDENTITY, data, off, torch.int32, path)
    ref = op.segreduce(red, op.MAP_IDENTITY, data, off, np.int32)
    assert np.count_nonzero(np.diff(off) == 0) > 100
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("dts", [(np.float32, np.float32), (np.float32, np.float64), (np.float64, np.float64),
                                 (np.int64, np.int64), (np.int64, np.int32), (np.int32, np.int32)])
def test_segreduce_dtypes(dts, path):
    din, dout = dts
    data, off = _seg_case(77, 2000, 0, 500, din)
    got = _segreduce_path(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, TORCH_DT[dout], path)
    if np.dtype(dout).kind == "i":
        ref = op.segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, dout)
        assert np.array_equal(got, ref)
    else:
        x = data.astype(np.float64)
        ref = op.segreduce_fast(op.RED_ADD, op.MAP_IDENTITY, (x * x + 1), off, np.float64)
        absum = op.segreduce_fast(op.RED_ADD, op.MAP_IDENTITY, np.abs(x * x + 1), off, np.float64)
        u = 2.0 ** -24 if dout == np.float32 or din == np.float32 else 2.0 ** -53
        n = np.maximum(np.diff(off), 1)
        assert np.all(np.abs(got - ref) <= 2 * n * u * absum + 1e-30)


def test_segreduce_scaled_sweep_size():
    # the HBM-sized workload: 2^20 segments, lengths U{0..256}; whole output compared
    data, lengths = synth.ragged_flat_int32(1, 1 << 20)
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    got = api.accel_segreduce(op.RED_ADD, op.MAP_SQ_PLUS_ONE, _t(data), _t(off), torch.int64).cpu().numpy()
    ref = op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, np.int64)
    assert np.array_equal(got, ref)


# --------------------------------------------------------------------------------- loop
# every output is compared: n = 100,001 and 100,003 are multiples of neither a warp, a CTA
# nor the grid stride, so the partial last warp and the grid-stride remainder are checked;
# n = 3 is a single partial warp
@pytest.mark.parametrize("n", [100_001, 100_003, 3])
@pytest.mark.parametrize("dt", [np.int32, np.int64, np.float32, np.float64])
@pytest.mark.parametrize("body", [op.LOOP_AXPY, op.LOOP_SCALE])
def test_loop_bodies(dt, body, n):
    g = synth.rng(2)
    if np.dtype(dt).kind == "i":
        a, b = g.integers(-1000, 1000, size=(2, n)).astype(dt)
    else:
        a, b = g.standard_normal((2, n)).astype(dt)
    t0 = _t(a)
    api.accel_loop(body, t0, _t(b), 2.0)
    ref = op.loop_body(body, a, b, 2)
    got = t0.cpu().numpy()
    assert got.shape == ref.shape
    if np.dtype(dt).kind == "i":
        assert np.array_equal(got, ref)
    else:
        # one multiply and one add in the element type: within 1 ulp of the float64 result
        np.testing.assert_allclose(got, ref, rtol=2 * np.finfo(dt).eps, atol=0)


def test_loop_leaves_elements_past_n_untouched():
    a = np.arange(1000, dtype=np.float32)
    b = np.ones(1000, dtype=np.float32)
    t0 = _t(a)
    api.accel_loop(op.LOOP_AXPY, t0, _t(b), 2.0, n=997)
    got = t0.cpu().numpy()
    np.testing.assert_array_equal(got[:997], a[:997] + 2)
    np.testing.assert_array_equal(got[997:], a[997:])
