"""Brute-force enumeration over HMM state paths (test infrastructure only).

An independent definition of the quantities the forward recursion and forward-backward
compute, used to pin :mod:`oracle.hmm` on tiny models (K^T paths):

    P(o)                 = sum over paths z of pi_{z_1} b_{z_1}(o_1) prod_{t>1} A_{z_{t-1} z_t} b_{z_t}(o_t)
    E[#(i->j)]           = sum_z P(z | o) * #{t : z_t = i, z_{t+1} = j}
    E[#(j emits k)]      = sum_z P(z | o) * #{t : z_t = j, o_t = k}
    E[z_1 = j]           = sum_z P(z | o) * [z_1 = j]

Pure Python loops over itertools.product; float64.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def path_probs(A, B, pi, obs):
    """Yield (path, joint probability P(z, o)) for every state path."""
    K = len(pi)
    T = len(obs)
    for z in itertools.product(range(K), repeat=T):
        p = pi[z[0]] * B[z[0]][obs[0]]
        for t in range(1, T):
            p *= A[z[t - 1]][z[t]] * B[z[t]][obs[t]]
        yield z, p


def loglik(A, B, pi, obs) -> float:
    return math.log(sum(p for _, p in path_probs(A, B, pi, obs)))


def expected_counts(A, B, pi, obs):
    """(logL, xi [K,K], counts [K,M], gamma_1 [K]) by enumeration."""
    K = len(pi)
    M = len(B[0])
    T = len(obs)
    paths = list(path_probs(A, B, pi, obs))
    Z = sum(p for _, p in paths)
    xi = np.zeros((K, K))
    cnt = np.zeros((K, M))
    g1 = np.zeros(K)
    for z, p in paths:
        w = p / Z
        for t in range(T - 1):
            xi[z[t], z[t + 1]] += w
        for t in range(T):
            cnt[z[t], obs[t]] += w
        g1[z[0]] += w
    return math.log(Z), xi, cnt, g1
