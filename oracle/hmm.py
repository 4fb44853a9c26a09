"""Oracle for the HMM workloads (test infrastructure only).

The paper (Expression Acceleration, arXiv 2211.00621) does not mention hidden Markov
models.  The HMM forward recursion is used as a synthetic program built from its pattern
vocabulary: for every time step t (a sequential loop, as the foldl of Listing 1), the new
forward vector is a ``map`` over states j of a ``reduce`` over states i (Appendix A,
Fig. "pmexpr-extension").  The arithmetic below is the textbook forward algorithm and
forward-backward expected counts, in float64, with these readings:

* natural logarithms; logL = log P(o_1 .. o_T);
* the first emission is included: alpha_1(j) = pi_j b_j(o_1);
* parameters enter as log-probabilities that are treated as free parameters (no row
  renormalisation inside the function), so d logL / d logA_ij is the expected number of
  i->j transitions and d logL / d logB_jk the expected number of times state j emits k.

Layouts: A[i, j] = P(z_{t+1}=j | z_t=i); B[j, k] = P(o_t=k | z_t=j); pi[j] = P(z_1=j).
The re-estimation functions at the end (softmax-parameterised gradient, Baum-Welch M-step)
are the textbook step after the expected counts.
"""
from __future__ import annotations

import numpy as np


def _lse(v: np.ndarray, axis=None):
    m = np.max(v, axis=axis, keepdims=True)
    r = m + np.log(np.sum(np.exp(v - m), axis=axis, keepdims=True))
    return np.squeeze(r, axis=axis) if axis is not None else float(r.reshape(()))


def forward_log(logA: np.ndarray, logB: np.ndarray, logpi: np.ndarray, obs: np.ndarray) -> float:
    """Log-space forward recursion.

    la_1(j) = log pi_j + log B[j, o_1]
    la_t(j) = LSE_i( la_{t-1}(i) + log A[i, j] ) + log B[j, o_t]
    logL    = LSE_j la_T(j)
    """
    la = logpi + logB[:, obs[0]]
    for t in range(1, len(obs)):
        la = _lse(la[:, None] + logA, axis=0) + logB[:, obs[t]]
    return _lse(la)


def forward_scaled(A: np.ndarray, B: np.ndarray, pi: np.ndarray, obs: np.ndarray,
                   return_all: bool = False):
    """Scaled forward recursion.

    a~_1 = pi o b(o_1);  a~_t = (a^_{t-1} A) o b(o_t);  c_t = sum_j a~_t(j);
    a^_t = a~_t / c_t;   logL = sum_t log c_t.
    With ``return_all`` also returns the normalised alphas [T, K] and the c_t [T].
    """
    T = len(obs)
    K = len(pi)
    ahat = np.empty((T, K)) if return_all else None
    c = np.empty(T)
    a = pi * B[:, obs[0]]
    c[0] = a.sum()
    a = a / c[0]
    if return_all:
        ahat[0] = a
    for t in range(1, T):
        a = (a @ A) * B[:, obs[t]]
        c[t] = a.sum()
        a = a / c[t]
        if return_all:
            ahat[t] = a
    logL = float(np.sum(np.log(c)))
    if return_all:
        return logL, ahat, c
    return logL


def backward_scaled(A: np.ndarray, B: np.ndarray, obs: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Scaled backward recursion matching :func:`forward_scaled`'s c_t.

    b^_T = 1;  b^_t = A ( b(o_{t+1}) o b^_{t+1} ) / c_{t+1}.   Returns [T, K].
    """
    T = len(obs)
    K = A.shape[0]
    bhat = np.empty((T, K))
    bhat[T - 1] = 1.0
    for t in range(T - 2, -1, -1):
        bhat[t] = A @ (B[:, obs[t + 1]] * bhat[t + 1]) / c[t + 1]
    return bhat


def expected_counts(A: np.ndarray, B: np.ndarray, pi: np.ndarray, obs: np.ndarray):
    """Forward-backward expected counts for one sequence.

    gamma_t(j)  = a^_t(j) b^_t(j)                              (posterior of z_t = j)
    xi(i, j)    = sum_{t<T} a^_t(i) A_ij b_j(o_{t+1}) b^_{t+1}(j) / c_{t+1}
    counts(j,k) = sum_t gamma_t(j) [o_t = k]
    Returns (logL, xi [K,K], counts [K,M], gamma_1 [K]); these are the gradients of logL
    with respect to log A, log B and log pi under the free-parameter reading.
    """
    logL, ahat, c = forward_scaled(A, B, pi, obs, return_all=True)
    bhat = backward_scaled(A, B, obs, c)
    T = len(obs)
    K, M = B.shape
    xi = np.zeros((K, K))
    for t in range(T - 1):
        w = B[:, obs[t + 1]] * bhat[t + 1] / c[t + 1]
        xi += np.outer(ahat[t], w)
    xi *= A
    gamma = ahat * bhat
    counts = np.zeros((K, M))
    for t in range(T):
        counts[:, obs[t]] += gamma[t]
    return logL, xi, counts, gamma[0].copy()


# ------------------------------------------------------------------------ batches
def loglik_batch(p: dict, seqs=None, log_space: bool = False, params: dict | None = None) -> np.ndarray:
    """logL for each sequence (or the listed subset) of a workload dict from synth.

    ``params`` overrides the float64 parameters (A, B, pi), e.g. with float32-rounded
    ones converted to float64.
    """
    q = params if params is not None else p
    obs, off = p["obs"], p["offsets"]
    idx = range(len(off) - 1) if seqs is None else seqs
    out = []
    for s in idx:
        o = obs[off[s]:off[s + 1]]
        if log_space:
            out.append(forward_log(np.log(q["A"]), np.log(q["B"]), np.log(q["pi"]), o))
        else:
            out.append(forward_scaled(q["A"], q["B"], q["pi"], o))
    return np.array(out)


def gradients_batch(p: dict, seqs=None, weights=None, params: dict | None = None):
    """Summed (optionally weighted) gradients of sum_s w_s logL_s over the sequences.

    Returns (logL [n], grad_logA [K,K], grad_logB [K,M], grad_logpi [K]).
    """
    q = params if params is not None else p
    obs, off = p["obs"], p["offsets"]
    idx = list(range(len(off) - 1)) if seqs is None else list(seqs)
    K, M = q["B"].shape
    gA, gB, gpi = np.zeros((K, K)), np.zeros((K, M)), np.zeros(K)
    lls = []
    for n, s in enumerate(idx):
        w = 1.0 if weights is None else float(weights[n])
        ll, xi, cnt, g1 = expected_counts(q["A"], q["B"], q["pi"], obs[off[s]:off[s + 1]])
        lls.append(ll)
        gA += w * xi
        gB += w * cnt
        gpi += w * g1
    return np.array(lls), gA, gB, gpi


def loglik_scaled_batch(p: dict, seqs=None, params: dict | None = None) -> np.ndarray:
    """logL of many sequences by the scaled recursion of :func:`forward_scaled`, all
    sequences advanced together: the forward vectors of the sequences still running at step t
    are the rows of one matrix X, and the step is one library matrix product X A (each row is
    that sequence's a^_{t-1} A, rows independent), then the emission o b(o_t) and the
    division of each row by its sum c_t; logL_s = sum_t log c_t.  Same arithmetic as the
    per-sequence loop, for sizes where that loop is too slow."""
    q = params if params is not None else p
    A, B, pi = q["A"], q["B"], q["pi"]
    obs, off = p["obs"], p["offsets"]
    idx = np.arange(len(off) - 1) if seqs is None else np.asarray(list(seqs), dtype=np.int64)
    T = (off[idx + 1] - off[idx]).astype(np.int64)
    order = np.argsort(-T, kind="stable")          # longest first: the running set is a prefix
    sidx, sT, start = idx[order], T[order], off[idx[order]]
    logL = np.zeros(len(sidx))
    x = pi[None, :] * B[:, obs[start]].T            # a~_1 = pi o b(o_1)
    for t in range(int(sT.max()) if len(sT) else 0):
        n = int(np.count_nonzero(sT > t))
        if t > 0:
            x = (x[:n] @ A) * B[:, obs[start[:n] + t]].T
        c = x.sum(axis=1)
        x = x / c[:, None]
        logL[:n] += np.log(c)
    out = np.empty(len(sidx))
    out[order] = logL
    return out


def params_from_f32_logs(logs: dict) -> dict:
    """float64 parameters equal to exp of the float32 log inputs (the kernel's inputs)."""
    return {"A": np.exp(logs["log_A"].astype(np.float64)),
            "B": np.exp(logs["log_B"].astype(np.float64)),
            "pi": np.exp(logs["log_pi"].astype(np.float64))}


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (8 significant bits) to nearest, ties to even, returned
    as float32: add half a bfloat16 unit (0x7FFF plus the kept part's lowest bit, so that ties
    go to the even neighbour) to the IEEE bit pattern and clear the 16 low bits.  Finite
    inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def params_bf16_from_f32_logs(logs: dict) -> dict:
    """The parameters as the BF16 tensor-core forward holds them: exp of the float32 logs
    rounded to float32, then to bfloat16 for A and B (its matrix operand and emission
    table); pi stays float32 (it enters the first vector in FP32).  float64 arrays."""
    def r32(v):
        return np.exp(v.astype(np.float64)).astype(np.float32)
    return {"A": round_bf16(r32(logs["log_A"])).astype(np.float64),
            "B": round_bf16(r32(logs["log_B"])).astype(np.float64),
            "pi": r32(logs["log_pi"]).astype(np.float64)}


# ------------------------------------------------------------------------ re-estimation
# The step after the adjoint in a training loop (textbook; not in the paper).  Each
# parameter is a set of rows that are probability vectors: the rows of A (over j), the rows
# of B (over k), and pi.  Both functions work on the last axis of their arguments.
def softmax_rows_grad(logP: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Gradient with respect to unconstrained row parameters theta with P = softmax(theta)
    along each row, given g = the gradient with respect to log P read as free parameters
    (what expected_counts and gradients_batch return).  log P_ij = theta_ij - LSE_j' theta_ij',
    so by the chain rule
        dL/dtheta_ij = g_ij - P_ij * sum_j' g_ij',     P = softmax of the row of logP.
    Rows of the result sum to zero (adding a constant to a row of theta changes nothing)."""
    P = np.exp(logP - _lse(logP, axis=-1)[..., None])
    return g - P * np.sum(g, axis=-1, keepdims=True)


def mstep_rows(g: np.ndarray, logP_old: np.ndarray) -> np.ndarray:
    """Baum-Welch re-estimation of row-stochastic parameters from their expected counts g:
        P_new_ij = g_ij / sum_j' g_ij',   returned as log P_new.
    A row whose counts sum to zero (no sequence visits the state) keeps log P_old."""
    s = np.sum(g, axis=-1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        new = np.log(g) - np.log(s)
    return np.where(s > 0, new, logP_old)
