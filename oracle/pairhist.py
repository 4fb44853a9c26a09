"""Oracle for the all-pairs angular histogram (test infrastructure only).

A map over point pairs of a bin lookup, reduced into a histogram: the two-point angular
correlation shape (tpacf) that the paper lists among its workloads (Table 1), here on
synthetic points.  For unit vectors p_i, p_j the separation enters through the dot product

    d = (x_i x_j + y_i y_j) + z_i z_j,

with every product and sum rounded to float32 (the bin decision is taken in the kernel's
precision, so the counts must match exactly), and the bin of a pair is the number of edges
e_k >= d of the descending edge list (cosines of increasing angles): bin 0 holds pairs
closer than the first edge, bin len(edges) pairs beyond the last one.  With one point set
the unordered pairs i < j are counted; with two, every pair (i in A, j in B).
"""
from __future__ import annotations

import numpy as np


def dots_f32(p: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """d between point p [3] and each row of Q [n, 3], in float32 as defined above."""
    p = p.astype(np.float32)
    Q = Q.astype(np.float32)
    return (p[0] * Q[:, 0] + p[1] * Q[:, 1]) + p[2] * Q[:, 2]


def bins_of(d: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Number of edges >= d for each d (edges strictly decreasing float32)."""
    e = np.asarray(edges, dtype=np.float32)
    # -e is ascending; e_k >= d  <=>  -e_k <= -d
    return np.searchsorted(-e, -d.astype(np.float32), side="right")


def pair_histogram(A: np.ndarray, edges: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
    """int64 histogram with len(edges) + 1 bins over the pairs described above."""
    nb = len(edges) + 1
    h = np.zeros(nb, dtype=np.int64)
    if B is None:
        for i in range(len(A) - 1):
            h += np.bincount(bins_of(dots_f32(A[i], A[i + 1:]), edges), minlength=nb)
    else:
        for i in range(len(A)):
            h += np.bincount(bins_of(dots_f32(A[i], B), edges), minlength=nb)
    return h
