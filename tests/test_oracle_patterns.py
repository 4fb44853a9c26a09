"""Pins for oracle.patterns against the paper's worked examples, closed forms, brute
force written as plain Python builtins, and invariants (CPU only)."""
import functools
import math
import operator

import numpy as np
import pytest

from oracle import patterns as P
from paper_2211_00621_gb300 import synth


def test_listing1_axpy_closed_form():
    # Listing 1: loop n (lam i. axpy 2 i) with axpy c i: t1[i] <- t1[i] + c*t2[i].
    t1 = np.array([1, -2, 3, 40], dtype=np.int64)
    t2 = np.array([4, 5, -6, 7], dtype=np.int64)
    out = P.loop_body(P.LOOP_AXPY, t1, t2, 2)
    assert out.tolist() == [9, 8, -9, 54]


def test_appendix_loop_b_equals_2a():
    # Appendix A: loop n f with f i = tensorSet b [i] (muli 2 (tensorGet a i)).
    a = np.arange(-5, 6, dtype=np.int32)
    b = np.zeros_like(a)
    assert P.loop_body(P.LOOP_SCALE, b, a, 2).tolist() == [2 * v for v in range(-5, 6)]
    af = np.linspace(-1, 1, 7)
    np.testing.assert_array_equal(P.loop_body(P.LOOP_SCALE, np.zeros(7), af, 2.0), 2 * af)


def test_listing1_computesum_reduce_equals_foldl_builtin():
    # Listing 1 computeSum: reduce addi 0 s (n >= 100) and foldl addi 0 s give the same sum.
    s = synth.ragged_int32(3, 1, 150, 150)[0]
    assert P.reduce_op(P.RED_ADD, s, np.int64) == sum(int(v) for v in s)


def test_reduce_muli_product():
    # Appendix A: accelerate (reduce muli 1 s) is the product of s.
    s = np.array([3, -2, 5, 7, 1, -1], dtype=np.int64)
    assert P.reduce_op(P.RED_MUL, s) == math.prod(s.tolist()) == 210


def test_listing2_map_reduce_closed_form():
    # Listing 2: f x = c * (g x) with g x = x + 1, then reduce addi 0 (map f s):
    # sum_x c (x + 1) = c (sum x + n), for c in [10, 20].
    s = synth.ragged_int32(7, 1, 500, 500)[0].astype(np.int64)
    for c in (10, 13, 20):
        mapped = P.map_op(P.MAP_IDENTITY, s, np.int64) + 1
        mapped = P.map_op(P.MAP_SCALE, mapped, np.int64, scalar=c)
        assert P.reduce_op(P.RED_ADD, mapped) == c * (int(s.sum()) + len(s))


def test_map2_addi_and_map_ops_builtin():
    # Appendix A: accelerate (map2 addi s1 s2) is the elementwise sum.
    s1 = np.array([1, 2, 3, -4], dtype=np.int32)
    s2 = np.array([10, -20, 30, 40], dtype=np.int32)
    assert P.map_op(P.MAP_ADD2, s1, np.int32, y=s2).tolist() == list(map(operator.add, s1.tolist(), s2.tolist()))
    assert P.map_op(P.MAP_MUL2, s1, np.int64, y=s2).tolist() == [10, -40, 90, -160]
    assert P.map_op(P.MAP_SQ_PLUS_ONE, s1, np.int64).tolist() == [2, 5, 10, 17]
    assert P.map_op(P.MAP_NEG, s1, np.int32).tolist() == [-1, -2, -3, 4]
    assert P.map_op(P.MAP_ABS, s1, np.int32).tolist() == [1, 2, 3, 4]
    # int64 arithmetic narrowed to int32 wraps (two's complement).
    assert P.map_op(P.MAP_SQ_PLUS_ONE, np.array([65536], dtype=np.int32), np.int32).tolist() == [1]


def test_reduce_min_max_neutral():
    x = np.array([5, -3, 9, 2], dtype=np.int64)
    assert P.reduce_op(P.RED_MIN, x) == min(x.tolist())
    assert P.reduce_op(P.RED_MAX, x) == max(x.tolist())
    e = np.array([], dtype=np.int64)
    assert P.reduce_op(P.RED_MAX, e) == np.iinfo(np.int64).min
    assert P.reduce_op(P.RED_ADD, e) == 0
    assert P.reduce_op(P.RED_MUL, e) == 1


def test_marshal_roundtrip_and_offsets():
    seqs = synth.ragged_int32(1, 50, 0, 12)
    flat, off = P.marshal_ragged(seqs)
    assert off[0] == 0 and off[-1] == sum(len(s) for s in seqs) == len(flat)
    assert np.all(np.diff(off) >= 0)
    # flatten is concatenation (Appendix A): compare with itertools-free builtin concatenation.
    assert flat.tolist() == functools.reduce(operator.add, (s.tolist() for s in seqs), [])
    back = P.unmarshal_ragged(flat, off)
    assert all(np.array_equal(a, b) for a, b in zip(seqs, back))


def test_marshal_records_roundtrip():
    b = synth.bodies(0, 33)
    aos = b["aos"].view(np.uint8).reshape(33, 16)
    fields = [(0, np.float32), (4, np.float32), (8, np.float32), (12, np.float32)]
    soa = P.marshal_records(aos, fields)
    for f in range(4):
        np.testing.assert_array_equal(soa[f], b["aos"][:, f])
    np.testing.assert_array_equal(P.unmarshal_records(soa, fields, 16), aos)


def _segreduce_builtin(seqs, f):
    return [sum(f(int(v)) for v in s) for s in seqs]


def test_segreduce_bruteforce_tiny():
    seqs = synth.ragged_int32(2, 40, 0, 9, -1000, 1000)
    flat, off = P.marshal_ragged(seqs)
    seg = P.segreduce(P.RED_ADD, P.MAP_SQ_PLUS_ONE, flat, off, np.int64)
    assert seg.tolist() == _segreduce_builtin(seqs, lambda v: v * v + 1)
    # empty segments give the neutral element 0
    assert all(seg[s] == 0 for s in range(40) if len(seqs[s]) == 0)
    assert any(len(s) == 0 for s in seqs)


def test_segreduce_identity_sum_of_segments_equals_total():
    # sum over segments of segment sums == reduce over the flattened mapped sequence.
    cfg = synth.CFG_SEGREDUCE
    seqs = synth.ragged_int32(cfg["seed"], 300, cfg["len_lo"], cfg["len_hi"])
    flat, off = P.marshal_ragged(seqs)
    seg = P.segreduce_fast(P.RED_ADD, P.MAP_SQ_PLUS_ONE, flat, off, np.int64)
    x = flat.astype(np.int64)
    assert int(seg.sum()) == int(np.sum(x * x + 1))
    m = P.reduce_op(P.RED_MAX, seg)
    assert all(m >= v for v in seg.tolist()) and m in seg.tolist()


def test_segreduce_fast_matches_loop_definition():
    seqs = synth.ragged_int32(5, 120, 0, 30)
    flat, off = P.marshal_ragged(seqs)
    for op in (P.RED_ADD, P.RED_MAX):
        for fm in (P.MAP_IDENTITY, P.MAP_SQ_PLUS_ONE):
            a = P.segreduce(op, fm, flat, off, np.int64)
            b = P.segreduce_fast(op, fm, flat, off, np.int64)
            np.testing.assert_array_equal(a, b)


def test_segreduce_min_mul_builtin():
    seqs = synth.ragged_int32(9, 25, 0, 5, -9, 9)
    flat, off = P.marshal_ragged(seqs)
    mn = P.segreduce(P.RED_MIN, P.MAP_IDENTITY, flat, off, np.int64)
    ml = P.segreduce(P.RED_MUL, P.MAP_IDENTITY, flat, off, np.int64)
    imax = np.iinfo(np.int64).max
    assert mn.tolist() == [min(s.tolist()) if len(s) else imax for s in seqs]
    assert ml.tolist() == [math.prod(s.tolist()) for s in seqs]


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_float_reduce_within_rounding(dt):
    x = synth.rng(4).standard_normal(1000).astype(dt)
    assert P.reduce_op(P.RED_ADD, x, np.float64) == pytest.approx(math.fsum(x.tolist()), rel=1e-12, abs=1e-12)


# ------------------------------------------------------------ two-level flatten (next row 3)
def _groups(seed, G=7):
    rng = np.random.default_rng(seed)
    out = []
    for g in range(G):
        n = int(rng.integers(0, 5))                       # empty groups included
        out.append([rng.integers(-50, 50, size=int(rng.integers(0, 9))).astype(np.int32) for _ in range(n)])
    return out


def test_marshal_nested_roundtrip_and_offsets():
    groups = _groups(4)
    flat, off, goff = P.marshal_nested(groups)
    back = P.unmarshal_nested(flat, off, goff)
    assert len(back) == len(groups)
    for a, b in zip(groups, back):
        assert len(a) == len(b) and all(np.array_equal(x, y) for x, y in zip(a, b))
    # the flat data is the concatenation of every sequence in order (reduce (++), Listing-1 style)
    assert np.array_equal(flat, functools.reduce(lambda u, v: np.concatenate([u, v]),
                                                 [s for g in groups for s in g], np.zeros(0, np.int32)))
    assert goff[-1] == len(off) - 1 and off[-1] == len(flat)


def test_nested_reduce_of_reduces_is_the_nested_python_sum():
    # map (lam g. reduce (+) 0 (map (lam s. reduce (+) 0 s) g)) via two segmented reduces
    groups = _groups(5, G=9)
    flat, off, goff = P.marshal_nested(groups)
    inner = P.segreduce(P.RED_ADD, P.MAP_IDENTITY, flat, off, np.int64)
    outer = P.segreduce(P.RED_ADD, P.MAP_IDENTITY, inner, goff, np.int64)
    expect = [sum(int(v) for s in g for v in s) for g in groups]
    assert outer.tolist() == expect
