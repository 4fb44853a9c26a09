"""Oracle for the parallel patterns (test infrastructure only).

Paper passages followed (Expression Acceleration, arXiv 2211.00621):

* Appendix A, Fig. "pmexpr-extension" and the text after it: ``map f s`` applies f to
  every element; ``map2 f s1 s2`` applies f elementwise to two sequences; ``reduce f ne s``
  folds s with f starting from ne; ``flatten`` concatenates the inner sequences of a
  two-dimensional sequence; ``loop n f`` calls f i once for every i in [0, n) in an
  undefined order.
* Appendix B "Dynamic Assumptions": reduce assumes f associative with ne its neutral
  element, so any evaluation order gives the same value (exact for integers).
* Sec. 5 (Evaluation, Futhark): the compiler always uses 64-bit integers, so integer
  maps and reductions here compute in int64.
* Sec. 3.3 "Marshaling": arguments of an accelerated binding are converted from the
  sequential representation to the backend format, and results back.  For a ragged
  sequence of sequences the backend format is the flattened data plus an int64 offsets
  array (exclusive scan of lengths); for a sequence of records it is one array per field.

Everything is a direct sequential definition; no blocking or reordering.
"""
from __future__ import annotations

import numpy as np

# Operator names mirror the library's fixed operator set.
MAP_IDENTITY, MAP_SQ_PLUS_ONE, MAP_NEG, MAP_ABS, MAP_SCALE, MAP_ADD2, MAP_MUL2 = range(7)
RED_ADD, RED_MUL, RED_MIN, RED_MAX = range(4)
LOOP_AXPY, LOOP_SCALE = range(2)

_INT = (np.int32, np.int64)


def _is_int(dt) -> bool:
    return np.dtype(dt) in (np.dtype(np.int32), np.dtype(np.int64))


# ------------------------------------------------------------------ marshal / flatten
def marshal_ragged(seqs: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """flatten (Fig. pmexpr-extension): concatenation in input order + int64 offsets.

    offsets[0] = 0, offsets[s+1] = offsets[s] + |seqs[s]| (Sec. 3.3 marshaling into the
    backend's flat format).
    """
    S = len(seqs)
    offsets = np.zeros(S + 1, dtype=np.int64)
    for s in range(S):
        offsets[s + 1] = offsets[s] + len(seqs[s])
    dt = seqs[0].dtype if S else np.int32
    flat = np.empty(int(offsets[S]), dtype=dt)
    for s in range(S):
        flat[offsets[s]:offsets[s + 1]] = seqs[s]
    return flat, offsets


def unmarshal_ragged(flat: np.ndarray, offsets: np.ndarray) -> list[np.ndarray]:
    """Inverse of :func:`marshal_ragged` (results converted back, Sec. 3.3)."""
    return [flat[offsets[s]:offsets[s + 1]].copy() for s in range(len(offsets) - 1)]


def marshal_nested(groups: list[list[np.ndarray]]) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """flatten applied twice, [[[T]]] -> (flat, sequence offsets, group offsets): the sequences
    of all groups in order, as :func:`marshal_ragged`, and goffsets[g+1] = goffsets[g] +
    (number of sequences in group g), indices into the sequence offsets."""
    seqs = [s for g in groups for s in g]
    flat, offsets = marshal_ragged(seqs)
    G = len(groups)
    goffsets = np.zeros(G + 1, dtype=np.int64)
    for g in range(G):
        goffsets[g + 1] = goffsets[g] + len(groups[g])
    return flat, offsets, goffsets


def unmarshal_nested(flat: np.ndarray, offsets: np.ndarray, goffsets: np.ndarray) -> list[list[np.ndarray]]:
    """Inverse of :func:`marshal_nested`."""
    seqs = unmarshal_ragged(flat, offsets)
    return [seqs[goffsets[g]:goffsets[g + 1]] for g in range(len(goffsets) - 1)]


def marshal_records(aos: np.ndarray, fields: list[tuple[int, np.dtype]]) -> list[np.ndarray]:
    """Records {l_i = e_i} (Fig. mexpr-ast) to one array per field (Sec. 3.3).

    ``aos`` is a uint8 array [n, record_bytes]; ``fields`` lists (byte offset, dtype).
    """
    out = []
    for off, dt in fields:
        w = np.dtype(dt).itemsize
        out.append(np.ascontiguousarray(aos[:, off:off + w]).view(dt).reshape(-1))
    return out


def unmarshal_records(soa: list[np.ndarray], fields: list[tuple[int, np.dtype]],
                      record_bytes: int) -> np.ndarray:
    """Inverse of :func:`marshal_records`; bytes outside every field are zero."""
    n = len(soa[0]) if soa else 0
    aos = np.zeros((n, record_bytes), dtype=np.uint8)
    for (off, dt), col in zip(fields, soa):
        w = np.dtype(dt).itemsize
        aos[:, off:off + w] = np.ascontiguousarray(col.astype(dt)).view(np.uint8).reshape(n, w)
    return aos


# ------------------------------------------------------------------------------ map
def map_scalar(op: int, x, y, scalar, out_dt):
    """One application of a map/map2 operator to Python scalars (int or float).

    Integer outputs compute in unbounded Python ints and wrap to the output width, which
    equals int64 two's-complement arithmetic narrowed to the output (Sec. 5: 64-bit ints).
    """
    if op == MAP_IDENTITY:
        r = x
    elif op == MAP_SQ_PLUS_ONE:
        r = x * x + 1
    elif op == MAP_NEG:
        r = -x
    elif op == MAP_ABS:
        r = abs(x)
    elif op == MAP_SCALE:
        r = scalar * x
    elif op == MAP_ADD2:
        r = x + y
    elif op == MAP_MUL2:
        r = x * y
    else:
        raise ValueError(op)
    if _is_int(out_dt):
        bits = np.dtype(out_dt).itemsize * 8
        r = int(r) & ((1 << bits) - 1)
        if r >= 1 << (bits - 1):
            r -= 1 << bits
        return r
    return float(r)


def map_op(op: int, x: np.ndarray, out_dt, y: np.ndarray | None = None,
           scalar: float = 0.0) -> np.ndarray:
    """``map f s`` / ``map2 f s1 s2`` (Fig. pmexpr-extension), element by element.

    Integer operands are taken as int64 (Sec. 5); float results are computed in float64
    and rounded once to the output type.  MAP_SCALE with an integer output uses the
    scalar truncated to an integer.
    """
    n = len(x)
    out = np.empty(n, dtype=out_dt)
    xi = x.tolist()
    yi = y.tolist() if y is not None else [0] * n
    sc = int(scalar) if _is_int(out_dt) else float(scalar)
    for k in range(n):
        out[k] = map_scalar(op, xi[k], yi[k], sc, out_dt)
    return out


# --------------------------------------------------------------------------- reduce
def neutral(op: int, dt):
    """Neutral element ne of each reduce operator (Appendix B: ne must be f's identity)."""
    if op == RED_ADD:
        return 0 if _is_int(dt) else 0.0
    if op == RED_MUL:
        return 1 if _is_int(dt) else 1.0
    if _is_int(dt):
        info = np.iinfo(dt)
        return int(info.max) if op == RED_MIN else int(info.min)
    return float("inf") if op == RED_MIN else float("-inf")


def combine(op: int, a, b, dt):
    """The associative operator f of ``reduce f ne s`` (addi, muli, min, max)."""
    if op == RED_ADD:
        r = a + b
    elif op == RED_MUL:
        r = a * b
    elif op == RED_MIN:
        r = a if a <= b else b
    elif op == RED_MAX:
        r = a if a >= b else b
    else:
        raise ValueError(op)
    if _is_int(dt):
        bits = np.dtype(dt).itemsize * 8
        r = int(r) & ((1 << bits) - 1)
        if r >= 1 << (bits - 1):
            r -= 1 << bits
    return r


def reduce_op(op: int, x: np.ndarray, dt=None):
    """``reduce f ne s`` as the sequential left fold ``foldl f ne s`` (Listing 1).

    Integers accumulate exactly (Python ints wrapped to the output width); floats in
    float64.
    """
    dt = dt if dt is not None else x.dtype
    acc = neutral(op, dt)
    for v in x.tolist():
        acc = combine(op, acc, v if _is_int(dt) else float(v), dt)
    return acc


def segreduce(op: int, fused_map: int, data: np.ndarray, offsets: np.ndarray, out_dt,
              scalar: float = 0.0) -> np.ndarray:
    """``map (lam s. reduce f ne (map g s))`` over a flattened sequence of sequences.

    seg[s] = fold over k in [offsets[s], offsets[s+1]) of g(data[k]); an empty segment
    gives ne (Appendix B).  The map g is applied in the output type (int64 for the
    integer workload, Sec. 5).
    """
    S = len(offsets) - 1
    out = np.empty(S, dtype=out_dt)
    vals = data.tolist()
    sc = int(scalar) if _is_int(out_dt) else float(scalar)
    for s in range(S):
        acc = neutral(op, out_dt)
        for k in range(int(offsets[s]), int(offsets[s + 1])):
            acc = combine(op, acc, map_scalar(fused_map, vals[k], 0, sc, out_dt), out_dt)
        out[s] = acc
    return out


def segreduce_fast(op: int, fused_map: int, data: np.ndarray, offsets: np.ndarray,
                   out_dt) -> np.ndarray:
    """Vectorised form of :func:`segreduce` for ADD/MAX with IDENTITY or SQ_PLUS_ONE maps.

    Used only at sizes where the scalar loop is too slow; pinned against
    :func:`segreduce` in the oracle tests.  Integer sums are exact in int64.
    """
    assert fused_map in (MAP_IDENTITY, MAP_SQ_PLUS_ONE) and op in (RED_ADD, RED_MAX)
    x = data.astype(np.int64) if _is_int(out_dt) else data.astype(np.float64)
    if fused_map == MAP_SQ_PLUS_ONE:
        x = x * x + 1
    S = len(offsets) - 1
    out = np.full(S, neutral(op, out_dt), dtype=out_dt)
    lengths = np.diff(offsets)
    nz = np.nonzero(lengths > 0)[0]
    if len(nz):
        starts = offsets[nz]
        if op == RED_ADD:
            out[nz] = np.add.reduceat(x, starts)
        else:
            out[nz] = np.maximum.reduceat(x, starts)
    return out


# ----------------------------------------------------------------------------- loop
def loop_body(body: int, t0: np.ndarray, t1: np.ndarray, scalar) -> np.ndarray:
    """``loop n f`` (Fig. pmexpr-extension) with the two fixed bodies, i = 0..n-1 in order.

    AXPY : t0[i] <- t0[i] + c * t1[i]   (Listing 1, axpy with c = 2)
    SCALE: t0[i] <- c * t1[i]           (the b = 2 * a loop of Appendix A)
    The order is irrelevant: neither body reads what another iteration writes.
    Integer tensors use the scalar truncated to an integer, in int64 (Sec. 5).
    """
    out = t0.copy()
    isint = _is_int(t0.dtype)
    c = int(scalar) if isint else float(scalar)
    for i in range(len(t0)):
        x = int(t0[i]) if isint else float(t0[i])
        y = int(t1[i]) if isint else float(t1[i])
        r = x + c * y if body == LOOP_AXPY else c * y
        if isint:
            bits = t0.dtype.itemsize * 8
            r = r & ((1 << bits) - 1)
            if r >= 1 << (bits - 1):
                r -= 1 << bits
        out[i] = r
    return out
