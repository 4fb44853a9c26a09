"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws random inputs and nothing else: it holds none of the arithmetic of
the parallel patterns or of the HMM / all-pairs workloads.  Every generator takes an
explicit seed and uses ``numpy.random.Generator(PCG64(seed))`` so both sides see
bit-identical inputs.

Workload shapes (the synthetic programs the pattern vocabulary of the paper's
Figure "pmexpr-extension" -- map, map2, reduce, flatten, loop -- is exercised on):

* ragged int32 sequences: lengths uniform in [len_lo, len_hi] inclusive, values uniform
  in [val_lo, val_hi] inclusive (4,096 sequences, lengths 0..256, values -1000..1000);
* HMM parameters: Dirichlet(1) rows for the transition and emission matrices, drawn as
  normalised Exp(1) variates in float64; a uniform initial distribution;
* observation sequences: i.i.d. uniform symbols; lengths fixed, uniform, or log-uniform
  (round(exp(U(ln lo, ln hi))) clamped to [lo, hi]);
* bodies for the all-pairs workload: positions uniform in [0,1)^3, masses uniform in
  [0.5, 1.5].
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------- ragged
def ragged_int32(seed: int, S: int, len_lo: int = 0, len_hi: int = 256,
                 val_lo: int = -1000, val_hi: int = 1000) -> list[np.ndarray]:
    """S int32 sequences with lengths U{len_lo..len_hi} and values U{val_lo..val_hi}."""
    g = rng(seed)
    lengths = g.integers(len_lo, len_hi + 1, size=S, dtype=np.int64)
    total = int(lengths.sum())
    values = g.integers(val_lo, val_hi + 1, size=total, dtype=np.int64).astype(np.int32)
    out, pos = [], 0
    for n in lengths.tolist():
        out.append(values[pos:pos + n])
        pos += n
    return out


def ragged_lengths(seed: int, S: int, len_lo: int = 0, len_hi: int = 256) -> np.ndarray:
    """Only the lengths of :func:`ragged_int32` (same stream, same first draw)."""
    return rng(seed).integers(len_lo, len_hi + 1, size=S, dtype=np.int64)


def ragged_flat_int32(seed: int, S: int, len_lo: int = 0, len_hi: int = 256,
                      val_lo: int = -1000, val_hi: int = 1000) -> tuple[np.ndarray, np.ndarray]:
    """Same draws as :func:`ragged_int32`, returned as (concatenated values, lengths)."""
    g = rng(seed)
    lengths = g.integers(len_lo, len_hi + 1, size=S, dtype=np.int64)
    total = int(lengths.sum())
    values = g.integers(val_lo, val_hi + 1, size=total, dtype=np.int64).astype(np.int32)
    return values, lengths


# -------------------------------------------------------------------------------- HMM
def dirichlet1_rows(g: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Rows drawn from Dirichlet(1,...,1) as normalised Exp(1) variates, float64."""
    e = g.exponential(1.0, size=(rows, cols))
    return e / e.sum(axis=1, keepdims=True)


def hmm_params(seed: int, K: int, M: int) -> dict:
    """Transition A [K,K], emission B [K,M] (rows Dirichlet(1)) and uniform pi [K], float64."""
    g = rng(seed)
    A = dirichlet1_rows(g, K, K)
    B = dirichlet1_rows(g, K, M)
    pi = np.full(K, 1.0 / K)
    return {"A": A, "B": B, "pi": pi}


def seq_lengths(seed: int, S: int, kind: str, lo: int, hi: int) -> np.ndarray:
    """Sequence lengths: 'fixed' (= hi), 'uniform' U{lo..hi}, 'loguniform' in [lo, hi]."""
    g = rng(seed)
    if kind == "fixed":
        return np.full(S, hi, dtype=np.int64)
    if kind == "uniform":
        return g.integers(lo, hi + 1, size=S, dtype=np.int64)
    if kind == "loguniform":
        x = np.exp(g.uniform(np.log(lo), np.log(hi), size=S))
        return np.clip(np.rint(x), lo, hi).astype(np.int64)
    raise ValueError(kind)


def observations(seed: int, lengths: np.ndarray, M: int) -> tuple[np.ndarray, np.ndarray]:
    """i.i.d. uniform symbols in [0, M) for each sequence: (flat int32 obs, int64 offsets)."""
    g = rng(seed)
    total = int(lengths.sum())
    obs = g.integers(0, M, size=total, dtype=np.int64).astype(np.int32)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    return obs, offsets


def hmm_workload(seed: int, K: int, M: int, S: int, kind: str, lo: int, hi: int) -> dict:
    """Parameters + observations for one HMM configuration (sub-streams seed, seed+1, seed+2)."""
    p = hmm_params(seed, K, M)
    lengths = seq_lengths(seed + 1, S, kind, lo, hi)
    obs, offsets = observations(seed + 2, lengths, M)
    p.update(obs=obs, offsets=offsets, lengths=lengths, K=K, M=M, S=S)
    return p


def hmm_log_inputs_f32(p: dict) -> dict:
    """The float32 log-space parameters handed to the library: roundings of the float64 ones."""
    return {
        "log_A": np.log(p["A"]).astype(np.float32),
        "log_B": np.log(p["B"]).astype(np.float32),
        "log_pi": np.log(p["pi"]).astype(np.float32),
    }


# ------------------------------------------------------------------------- all-pairs
def bodies(seed: int, N: int) -> dict:
    """N bodies: positions U[0,1)^3 and masses U[0.5,1.5], float64 and their float32 roundings.

    ``aos`` is the record array {pos: float3, mass: float} as 16-byte float32 records.
    """
    g = rng(seed)
    pos = g.random((N, 3))
    mass = g.uniform(0.5, 1.5, size=N)
    aos = np.empty((N, 4), dtype=np.float32)
    aos[:, :3] = pos.astype(np.float32)
    aos[:, 3] = mass.astype(np.float32)
    return {"pos": pos, "mass": mass, "aos": aos}


# ----------------------------------------------------------- angular pair histogram
def sphere_points(seed: int, N: int) -> np.ndarray:
    """N points uniform on the unit sphere (normalised Gaussian vectors), float32 [N, 3]."""
    g = rng(seed)
    v = g.normal(size=(N, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


def angle_edges(nbins: int, amin_arcmin: float, amax_arcmin: float) -> np.ndarray:
    """nbins + 1 bin edges for angular separations log-spaced between amin and amax
    arcminutes, given as their cosines (float32, strictly decreasing)."""
    k = np.arange(nbins + 1, dtype=np.float64)
    theta = amin_arcmin * (amax_arcmin / amin_arcmin) ** (k / nbins) * (np.pi / (180.0 * 60.0))
    return np.cos(theta).astype(np.float32)


# ------------------------------------------------------------------------ configs
# The five workload configurations, by what they are.
CFG_SEGREDUCE = dict(seed=0, S=4096, len_lo=0, len_hi=256, val_lo=-1000, val_hi=1000)
CFG_HMM_PLAIN = dict(seed=0, K=64, M=32, S=512, kind="fixed", lo=1000, hi=1000)
CFG_HMM_BATCHED = dict(seed=0, K=256, M=64, S=4096, kind="loguniform", lo=50, hi=5000)
CFG_HMM_ADJOINT = dict(seed=0, K=256, M=64, S=1024, kind="uniform", lo=200, hi=2000)
CFG_ALLPAIRS = dict(seed=0, N=65536, eps=1e-3)
# few, very long sequences (the parallel-in-T forward); beside the hot-path rows, not in their step
CFG_HMM_LONG = dict(seed=0, K=64, M=32, S=4, kind="fixed", lo=250000, hi=250000)
# all-pairs angular histogram (tpacf shape): 20 log-spaced bins from 1 to 10,000 arcminutes
CFG_PAIRHIST = dict(seed=0, N=32768, nbins=20, amin=1.0, amax=10000.0)
