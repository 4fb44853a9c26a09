"""Oracle for the all-pairs map-of-reduce (test infrastructure only).

A map over bodies i of a reduce over bodies j (Appendix A, Fig. "pmexpr-extension":
``map`` of ``reduce addi``), on a sequence of records {pos: float3, mass: float}.  The
paper's own workloads of this shape are tpacf and mri-q (Table 1); the arithmetic here is
softened gravity with G = 1, in float64:

    a_i = sum_j m_j (p_j - p_i) / (|p_j - p_i|^2 + eps^2)^(3/2)

Readings: eps is a length (eps^2 is added to r^2); the j = i term is included and is zero.
"""
from __future__ import annotations

import numpy as np


def accel_one(pos: np.ndarray, mass: np.ndarray, i: int, eps: float) -> np.ndarray:
    """a_i for one body, summing over every j (including j = i)."""
    d = pos - pos[i]
    r2 = np.sum(d * d, axis=1) + eps * eps
    w = mass / (r2 * np.sqrt(r2))
    return np.sum(w[:, None] * d, axis=0)


def accel(pos: np.ndarray, mass: np.ndarray, eps: float, idx=None) -> np.ndarray:
    """a_i for every body (or the listed subset), [n, 3] float64."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    ids = range(len(mass)) if idx is None else idx
    return np.array([accel_one(pos, mass, int(i), eps) for i in ids]).reshape(-1, 3)


def term_scale(pos: np.ndarray, mass: np.ndarray, eps: float, idx) -> np.ndarray:
    """sum_j |term_ij| / sqrt(N) per listed body: the scale of the sum's rounding error."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    out = []
    for i in idx:
        d = pos - pos[int(i)]
        r2 = np.sum(d * d, axis=1) + eps * eps
        out.append(np.sum(mass * np.sqrt(np.sum(d * d, axis=1)) / (r2 * np.sqrt(r2))))
    return np.array(out) / np.sqrt(len(mass))
