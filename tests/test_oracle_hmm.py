"""Pins for oracle.hmm: brute force over all state paths, closed forms, invariants and
central finite differences (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import brute, hmm
from paper_2211_00621_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name + ".json")) as f:
        c = json.load(f)
    return {k: np.array(v) if k not in ("source",) else v for k, v in c.items()}


@pytest.mark.parametrize("name", ["hmm_k2_t5", "hmm_k3_t4"])
def test_forward_matches_bruteforce_fixture(name):
    c = _load(name)
    obs = c["obs"].astype(np.int64)
    ll_s = hmm.forward_scaled(c["A"], c["B"], c["pi"], obs)
    ll_l = hmm.forward_log(np.log(c["A"]), np.log(c["B"]), np.log(c["pi"]), obs)
    assert ll_s == pytest.approx(float(c["loglik"]), rel=1e-13)
    assert ll_l == pytest.approx(float(c["loglik"]), rel=1e-13)


@pytest.mark.parametrize("name", ["hmm_k2_t5", "hmm_k3_t4"])
def test_expected_counts_match_bruteforce_fixture(name):
    c = _load(name)
    ll, xi, cnt, g1 = hmm.expected_counts(c["A"], c["B"], c["pi"], c["obs"].astype(np.int64))
    np.testing.assert_allclose(xi, c["xi"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(cnt, c["counts"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g1, c["gamma1"], rtol=1e-12, atol=1e-14)


def test_bruteforce_random_k2_t5():
    p = synth.hmm_workload(11, 2, 4, 3, "fixed", 5, 5)
    for s in range(3):
        o = p["obs"][p["offsets"][s]:p["offsets"][s + 1]]
        ref = brute.loglik(p["A"], p["B"], p["pi"], o)
        assert hmm.forward_scaled(p["A"], p["B"], p["pi"], o) == pytest.approx(ref, rel=1e-14)
        assert hmm.forward_log(np.log(p["A"]), np.log(p["B"]), np.log(p["pi"]), o) == pytest.approx(ref, rel=1e-14)


def test_closed_form_uniform_emissions():
    # b_j(o) = 1/M for all j, o: logL = -T log M whatever A and pi are.
    K, M, T = 5, 7, 40
    g = synth.rng(1)
    A = synth.dirichlet1_rows(g, K, K)
    pi = synth.dirichlet1_rows(g, 1, K)[0]
    B = np.full((K, M), 1.0 / M)
    o = g.integers(0, M, T)
    assert hmm.forward_scaled(A, B, pi, o) == pytest.approx(-T * math.log(M), rel=1e-13)
    assert hmm.forward_log(np.log(A), np.log(B), np.log(pi), o) == pytest.approx(-T * math.log(M), rel=1e-13)


def test_closed_form_single_state():
    # K = 1: logL = sum_t log B(o_t).
    B = np.array([[0.1, 0.2, 0.3, 0.4]])
    o = np.array([3, 0, 0, 2, 1, 3])
    ref = sum(math.log(B[0, k]) for k in o)
    assert hmm.forward_scaled(np.ones((1, 1)), B, np.ones(1), o) == pytest.approx(ref, rel=1e-14)


def test_closed_form_identity_transitions():
    # A = I: the state never changes, logL = log sum_j pi_j prod_t b_j(o_t).
    K, M, T = 4, 3, 12
    g = synth.rng(2)
    B = synth.dirichlet1_rows(g, K, M)
    pi = synth.dirichlet1_rows(g, 1, K)[0]
    o = g.integers(0, M, T)
    ref = math.log(sum(pi[j] * math.prod(B[j, k] for k in o) for j in range(K)))
    assert hmm.forward_scaled(np.eye(K), B, pi, o) == pytest.approx(ref, rel=1e-13)


def test_closed_form_rows_equal_pi():
    # Every row of A equal to pi: the z_t are i.i.d. pi, logL = sum_t log sum_j pi_j b_j(o_t).
    K, M, T = 6, 5, 30
    g = synth.rng(3)
    B = synth.dirichlet1_rows(g, K, M)
    pi = synth.dirichlet1_rows(g, 1, K)[0]
    A = np.tile(pi, (K, 1))
    o = g.integers(0, M, T)
    ref = sum(math.log(float(np.dot(pi, B[:, k]))) for k in o)
    assert hmm.forward_scaled(A, B, pi, o) == pytest.approx(ref, rel=1e-13)


def test_scaled_equals_logspace_medium():
    p = synth.hmm_workload(0, 64, 32, 2, "fixed", 300, 300)
    a = hmm.loglik_batch(p)
    b = hmm.loglik_batch(p, log_space=True)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_expected_counts_invariants():
    p = synth.hmm_workload(5, 8, 6, 4, "uniform", 5, 30)
    lls, gA, gB, gpi = hmm.gradients_batch(p)
    L = p["lengths"]
    assert gA.sum() == pytest.approx(float(np.sum(L - 1)), rel=1e-12)
    assert gB.sum() == pytest.approx(float(np.sum(L)), rel=1e-12)
    assert gpi.sum() == pytest.approx(4.0, rel=1e-12)
    assert (gA >= 0).all() and (gB >= 0).all() and (gpi >= 0).all()
    # counts of symbol k over states equal the number of times k was observed
    np.testing.assert_allclose(gB.sum(axis=0), np.bincount(p["obs"], minlength=6), rtol=1e-12)


def test_gradients_equal_central_finite_differences():
    # d logL / d logA_ij (free log parameters) by central differences, h = 1e-6, float64.
    p = synth.hmm_workload(8, 4, 3, 2, "fixed", 12, 12)
    _, gA, gB, gpi = hmm.gradients_batch(p)
    lA, lB, lpi = np.log(p["A"]), np.log(p["B"]), np.log(p["pi"])
    obs, off = p["obs"], p["offsets"]

    def total(lA_, lB_, lpi_):
        return sum(hmm.forward_log(lA_, lB_, lpi_, obs[off[s]:off[s + 1]]) for s in range(2))

    h = 1e-6
    for (i, j) in [(0, 0), (1, 3), (3, 2), (2, 1)]:
        a, b = lA.copy(), lA.copy()
        a[i, j] += h
        b[i, j] -= h
        fd = (total(a, lB, lpi) - total(b, lB, lpi)) / (2 * h)
        assert fd == pytest.approx(gA[i, j], rel=1e-6, abs=1e-6)
    for (j, k) in [(0, 0), (2, 1), (3, 2)]:
        a, b = lB.copy(), lB.copy()
        a[j, k] += h
        b[j, k] -= h
        fd = (total(lA, a, lpi) - total(lA, b, lpi)) / (2 * h)
        assert fd == pytest.approx(gB[j, k], rel=1e-6, abs=1e-6)
    for j in range(4):
        a, b = lpi.copy(), lpi.copy()
        a[j] += h
        b[j] -= h
        fd = (total(lA, lB, a) - total(lA, lB, b)) / (2 * h)
        assert fd == pytest.approx(gpi[j], rel=1e-6, abs=1e-6)


def test_bruteforce_expected_counts_random():
    p = synth.hmm_workload(21, 2, 3, 1, "fixed", 5, 5)
    o = p["obs"]
    ll, xi, cnt, g1 = brute.expected_counts(p["A"], p["B"], p["pi"], o)
    ll2, xi2, cnt2, g12 = hmm.expected_counts(p["A"], p["B"], p["pi"], o)
    assert ll2 == pytest.approx(ll, rel=1e-14)
    np.testing.assert_allclose(xi2, xi, rtol=1e-12)
    np.testing.assert_allclose(cnt2, cnt, rtol=1e-12)
    np.testing.assert_allclose(g12, g1, rtol=1e-12)


# ---------------------------------------------------------------- re-estimation (next row)
def _softmax(x):
    e = np.exp(x - x.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def _small_problem(seed, K=3, M=4, lens=(5, 4, 6)):
    rng = np.random.default_rng(seed)
    th = {"A": rng.normal(size=(K, K)), "B": rng.normal(size=(K, M)), "pi": rng.normal(size=K)}
    obs = [rng.integers(0, M, size=n) for n in lens]
    return th, obs


def _L_of_theta(th, obs):
    A, B, pi = _softmax(th["A"]), _softmax(th["B"]), _softmax(th["pi"])
    return sum(hmm.forward_log(np.log(A), np.log(B), np.log(pi), o) for o in obs)


def _counts(P, obs):
    K, M = P["B"].shape
    gA, gB, gpi = np.zeros((K, K)), np.zeros((K, M)), np.zeros(K)
    for o in obs:
        _, xi, cnt, g1 = hmm.expected_counts(P["A"], P["B"], P["pi"], o)
        gA += xi
        gB += cnt
        gpi += g1
    return gA, gB, gpi


def test_softmax_gradient_matches_central_differences():
    # L(theta) through the log-space forward (a path that shares nothing with the counts)
    th, obs = _small_problem(3)
    P = {k: _softmax(v) for k, v in th.items()}
    gA, gB, gpi = _counts(P, obs)
    an = {"A": hmm.softmax_rows_grad(th["A"], gA), "B": hmm.softmax_rows_grad(th["B"], gB),
          "pi": hmm.softmax_rows_grad(th["pi"], gpi)}
    h = 1e-5
    for name in ("A", "B", "pi"):
        fd = np.zeros_like(th[name])
        for idx in np.ndindex(th[name].shape):
            tp = {k: v.copy() for k, v in th.items()}
            tm = {k: v.copy() for k, v in th.items()}
            tp[name][idx] += h
            tm[name][idx] -= h
            fd[idx] = (_L_of_theta(tp, obs) - _L_of_theta(tm, obs)) / (2 * h)
        np.testing.assert_allclose(an[name], fd, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(an[name].sum(axis=-1), 0.0, atol=1e-12)   # row-shift invariance


def test_mstep_single_state_is_empirical_symbol_frequencies():
    # K = 1: the maximum-likelihood emission row is the symbol histogram, A and pi are 1
    rng = np.random.default_rng(5)
    M = 6
    obs = [rng.integers(0, M, size=n) for n in (7, 3, 11)]
    P = {"A": np.ones((1, 1)), "B": _softmax(rng.normal(size=(1, M))), "pi": np.ones(1)}
    gA, gB, gpi = _counts(P, obs)
    allobs = np.concatenate(obs)
    hist = np.bincount(allobs, minlength=M) / len(allobs)
    with np.errstate(divide="ignore"):
        np.testing.assert_allclose(hmm.mstep_rows(gB, np.log(P["B"])), np.log(hist)[None, :], rtol=1e-13)
    np.testing.assert_allclose(hmm.mstep_rows(gA, np.zeros((1, 1))), 0.0, atol=1e-15)
    np.testing.assert_allclose(hmm.mstep_rows(gpi, np.zeros(1)), 0.0, atol=1e-15)
    assert gA[0, 0] == pytest.approx(sum(len(o) - 1 for o in obs), rel=1e-13)


def test_mstep_does_not_decrease_the_likelihood():
    # Baum-Welch is an EM algorithm: every re-estimation step keeps or raises sum logL
    th, obs = _small_problem(11, K=4, M=5, lens=(9, 6, 12, 5))
    logP = {k: np.log(_softmax(v)) for k, v in th.items()}
    prev = None
    for _ in range(4):
        P = {k: np.exp(v) for k, v in logP.items()}
        L = sum(hmm.forward_log(logP["A"], logP["B"], logP["pi"], o) for o in obs)
        if prev is not None:
            assert L >= prev - 1e-10
        prev = L
        gA, gB, gpi = _counts(P, obs)
        logP = {"A": hmm.mstep_rows(gA, logP["A"]), "B": hmm.mstep_rows(gB, logP["B"]),
                "pi": hmm.mstep_rows(gpi, logP["pi"])}
        for v in logP.values():
            np.testing.assert_allclose(np.exp(v).sum(axis=-1), 1.0, rtol=1e-13)


def test_mstep_row_without_counts_keeps_its_parameters():
    g = np.array([[1.0, 3.0, 0.0], [0.0, 0.0, 0.0]])
    old = np.log(np.array([[0.2, 0.3, 0.5], [0.1, 0.6, 0.3]]))
    new = hmm.mstep_rows(g, old)
    np.testing.assert_allclose(new[1], old[1])
    np.testing.assert_allclose(new[0, :2], np.log([0.25, 0.75]), rtol=1e-15)
    assert new[0, 2] == -np.inf


# ------------------------------------------------------- sequence-batched scaled forward
@pytest.mark.parametrize("name", ["hmm_k2_t5", "hmm_k3_t4"])
def test_batched_forward_matches_bruteforce_fixture(name):
    c = _load(name)
    obs = c["obs"].astype(np.int32)
    p = {"A": c["A"], "B": c["B"], "pi": c["pi"], "obs": obs, "offsets": np.array([0, len(obs)], np.int64)}
    assert hmm.loglik_scaled_batch(p)[0] == pytest.approx(float(c["loglik"]), rel=1e-13)


def test_batched_forward_matches_brute_force_on_mixed_lengths():
    # brute force over every state path for each of several sequences of different lengths
    # (1 .. 6 steps), all advanced together by the batched form
    p = synth.hmm_workload(5, 2, 3, 12, "uniform", 1, 6)
    ll = hmm.loglik_scaled_batch(p)
    for s in range(12):
        o = p["obs"][p["offsets"][s]:p["offsets"][s + 1]]
        assert ll[s] == pytest.approx(brute.loglik(p["A"], p["B"], p["pi"], o), rel=1e-13)


@pytest.mark.parametrize("K,M,S,kind,lo,hi", [(7, 5, 40, "uniform", 1, 60), (64, 16, 30, "loguniform", 1, 500),
                                              (256, 64, 12, "loguniform", 50, 400)])
def test_batched_forward_matches_per_sequence_forward(K, M, S, kind, lo, hi):
    p = synth.hmm_workload(K + S, K, M, S, kind, lo, hi)
    ll = hmm.loglik_scaled_batch(p)
    ref = hmm.loglik_batch(p, log_space=True)        # the log-space recursion (no shared step)
    np.testing.assert_allclose(ll, ref, rtol=1e-12)
    sub = [S - 1, 0, 3]
    np.testing.assert_allclose(hmm.loglik_scaled_batch(p, seqs=sub), ref[sub], rtol=1e-12)


def test_batched_forward_closed_form_uniform_emissions():
    p = synth.hmm_workload(9, 6, 5, 20, "uniform", 1, 80)
    p["B"] = np.full((6, 5), 0.2)
    np.testing.assert_allclose(hmm.loglik_scaled_batch(p), -np.diff(p["offsets"]) * math.log(5), rtol=1e-13)


# ------------------------------------------------------------------- bfloat16 rounding
def test_round_bf16_hand_worked():
    # bfloat16 keeps 8 significant bits: the unit in the last place at 1.0 is 2^-7
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, 3.0, -1 - 3 * 2.0 ** -8,
                  2.0 ** -130], np.float32)
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 3.0, -1 - 2.0 ** -6, 2.0 ** -130], np.float32)
    # ties to even: 1 + 2^-8 is halfway between 1 (even) and 1 + 2^-7; 1 + 3 2^-8 halfway
    # between 1 + 2^-7 (odd) and 1 + 2^-6; just above the halfway point rounds up
    np.testing.assert_array_equal(hmm.round_bf16(x), want)


def test_round_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    g = synth.rng(8)
    x = np.concatenate([g.standard_normal(20000), np.exp(g.uniform(-30, 5, 20000)),
                        # exact halfway points: a bfloat16 value plus half its unit in the last place
                        (g.integers(1, 255, 2000) * 2.0 + 1) * 2.0 ** -9]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(hmm.round_bf16(x), ref)


def test_bf16_parameters_are_the_rounded_exponentials():
    p = synth.hmm_workload(2, 16, 8, 1, "fixed", 5, 5)
    logs = synth.hmm_log_inputs_f32(p)
    q = hmm.params_bf16_from_f32_logs(logs)
    # every entry has at most 8 significant bits and lies within half a bfloat16 unit
    for k, lk in (("A", "log_A"), ("B", "log_B")):
        v = q[k]
        m, _ = np.frexp(v)
        assert np.all(m * 2 ** 8 == np.round(m * 2 ** 8))
        ex = np.exp(logs[lk].astype(np.float64))
        assert np.all(np.abs(v - ex) <= 2.0 ** -8 * ex * (1 + 1e-6))
    np.testing.assert_array_equal(q["pi"], np.exp(logs["log_pi"].astype(np.float64)).astype(np.float32))
