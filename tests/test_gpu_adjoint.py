"""GPU parity of the HMM adjoint (hmm_adjoint and the HMMLogLik autograd function) with
the float64 oracle's forward-backward expected counts, brute-force enumeration and central
finite differences of the float64 forward.

Tolerance, entry by entry, against the oracle on the same float32-rounded log parameters
the kernels receive: |g - r| <= 1e-4 |r| + 1e-6 (row total of r).  Every gradient entry is
a sum of non-negative terms (expected counts), each formed with FP32 relative error, so
the error is relative to the entry; the row-total term only absorbs entries whose terms
underflow.  A wrong entry in a rarely visited state's row fails it, which a whole-matrix
norm would hide.  The relative Frobenius error is printed as a summary.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2211_00621_gb300 import _lib, api, synth
from oracle import hmm as ohmm

pytestmark = pytest.mark.gpu
DEV = "cuda"
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dev(p):
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    return logs, t, torch.from_numpy(p["obs"]).to(DEV), torch.from_numpy(p["offsets"]).to(DEV)


def _rel_fro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _check_grads(got, ref, rtol=1e-4, row_atol=1e-6):
    for g, r, name in zip(got, ref, ("log_A", "log_B", "log_pi")):
        g = np.asarray(g, dtype=np.float64)
        r = np.asarray(r, dtype=np.float64)
        tot = r.sum(axis=-1, keepdims=True)               # expected visits of the row's state
        err = np.abs(g - r)
        bad = err > rtol * np.abs(r) + row_atol * tot
        rel = err / np.maximum(np.abs(r), 1e-300)
        print(f"[adjoint {name}] max entry rel err {rel.max():.3e}, relative Frobenius {_rel_fro(g, r):.3e}")
        assert not bad.any(), (f"{name}: {int(bad.sum())} entries out of tolerance, worst at "
                               f"{np.unravel_index(np.argmax(err - rtol * np.abs(r) - row_atol * tot), r.shape)}")


@pytest.mark.parametrize("name", ["hmm_k2_t5", "hmm_k3_t4"])
def test_bruteforce_fixture(name):
    with open(os.path.join(GOLD, name + ".json")) as f:
        c = json.load(f)
    lA = torch.tensor(np.log(c["A"]), dtype=torch.float32, device=DEV)
    lB = torch.tensor(np.log(c["B"]), dtype=torch.float32, device=DEV)
    lpi = torch.tensor(np.log(c["pi"]), dtype=torch.float32, device=DEV)
    obs = torch.tensor(c["obs"], dtype=torch.int32, device=DEV)
    off = torch.tensor([0, len(c["obs"])], dtype=torch.int64, device=DEV)
    gA, gB, gpi, ll = api.hmm_adjoint(lA, lB, lpi, obs, off)
    np.testing.assert_allclose(gA.cpu().numpy(), c["xi"], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(gB.cpu().numpy(), c["counts"], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(gpi.cpu().numpy(), c["gamma1"], rtol=2e-5, atol=1e-6)
    assert abs(ll.item() - c["loglik"]) <= 1e-5 * abs(c["loglik"])


# K in {64, 128, 256} with a small enough emission table take the cluster kernels and the
# tensor-core count accumulation (emission counts there up to 256 padded symbols, else the
# SIMT count kernel); other shapes take the streaming kernels.  S = 200 and 1500 give
# cluster groups of 2-3 and 15-16 sequences.  With plans (S <= 32 pairs' worth), a round's
# backward and the next round's recomputation share a launch: side by side on disjoint CTA
# pairs when both fit (S = 200, 1500), else each on all pairs one after the other
# (S = 2400 on 76 pairs); S = 3000 has no plans (separate launches, groups by position).
@pytest.mark.parametrize("K,M,S,lo,hi", [(8, 5, 20, 1, 50), (37, 11, 13, 1, 130), (64, 32, 9, 100, 400),
                                         (64, 7, 40, 1, 200), (128, 200, 10, 20, 120), (64, 300, 6, 1, 90),
                                         (256, 100, 5, 30, 90), (256, 200, 6, 20, 80), (128, 16, 35, 1, 60),
                                         (64, 8, 200, 5, 60), (64, 8, 1500, 2, 12), (64, 8, 2400, 20, 60),
                                         (64, 8, 3000, 2, 12)])
def test_small_models_against_oracle(K, M, S, lo, hi):
    p = synth.hmm_workload(K * 3 + S, K, M, S, "uniform", lo, hi)
    logs, t, obs, off = _dev(p)
    w = synth.rng(5).uniform(0.5, 2.0, size=S)
    gA, gB, gpi, ll = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off,
                                      weights=torch.from_numpy(w).to(DEV))
    par = ohmm.params_from_f32_logs(logs)
    lls, rA, rB, rpi = ohmm.gradients_batch(p, weights=w, params=par)
    _check_grads((gA.cpu().numpy(), gB.cpu().numpy(), gpi.cpu().numpy()), (rA, rB, rpi))
    assert np.max(np.abs(ll.cpu().numpy() - lls) / np.abs(lls)) <= 1e-5


def test_config_shapes_subset_against_oracle():
    c = synth.CFG_HMM_ADJOINT
    p = synth.hmm_workload(c["seed"] + 7, c["K"], c["M"], 24, c["kind"], c["lo"], c["hi"])
    logs, t, obs, off = _dev(p)
    gA, gB, gpi, ll = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    lls, rA, rB, rpi = ohmm.gradients_batch(p, params=ohmm.params_from_f32_logs(logs))
    _check_grads((gA.cpu().numpy(), gB.cpu().numpy(), gpi.cpu().numpy()), (rA, rB, rpi))


def test_config_full_size_invariants_and_weighted_subset():
    c = synth.CFG_HMM_ADJOINT
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
    logs, t, obs, off = _dev(p)
    L = p["lengths"]
    gA, gB, gpi, ll = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    gA, gB, gpi = gA.cpu().numpy().astype(np.float64), gB.cpu().numpy().astype(np.float64), gpi.cpu().numpy()
    # one transition per step, one emission per step, one initial state per sequence
    assert abs(gA.sum() - np.sum(L - 1)) <= 1e-4 * np.sum(L - 1)
    assert abs(gB.sum() - np.sum(L)) <= 1e-4 * np.sum(L)
    assert abs(gpi.sum() - c["S"]) <= 1e-4 * c["S"]
    np.testing.assert_allclose(gB.sum(axis=0), np.bincount(p["obs"], minlength=c["M"]), rtol=1e-4)
    assert (gA >= 0).all() and (gB >= 0).all() and (gpi >= 0).all()
    # linearity in the weights: 0/1 weights select a subset, compared with the oracle
    sub = sorted(set(synth.rng(3).choice(c["S"], size=6, replace=False).tolist() + [int(np.argmax(L))]))
    w = np.zeros(c["S"])
    w[sub] = 1.0
    sA, sB, spi, _ = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off,
                                     weights=torch.from_numpy(w).to(DEV))
    _, rA, rB, rpi = ohmm.gradients_batch(p, seqs=sub, params=ohmm.params_from_f32_logs(logs))
    _check_grads((sA.cpu().numpy(), sB.cpu().numpy(), spi.cpu().numpy()), (rA, rB, rpi))
    # the forward's logL agrees with the FP32 log-space kernel
    ll2 = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off).cpu().numpy()
    assert np.max(np.abs(ll.cpu().numpy() - ll2) / np.abs(ll2)) <= 1e-5


def test_central_finite_differences_fp64():
    # d/d log A_ij and d/d log B_jk of sum_s logL_s by central differences (h = 1e-6) of the
    # float64 forward, on a few sequences of the adjoint configuration's model.
    c = synth.CFG_HMM_ADJOINT
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], 3, "uniform", 200, 400)
    logs, t, obs, off = _dev(p)
    gA, gB, gpi, _ = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    gA, gB = gA.cpu().numpy(), gB.cpu().numpy()
    lA = logs["log_A"].astype(np.float64)
    lB = logs["log_B"].astype(np.float64)
    lpi = logs["log_pi"].astype(np.float64)
    o, of = p["obs"], p["offsets"]

    def total(a, b):
        return sum(ohmm.forward_log(a, b, lpi, o[of[s]:of[s + 1]]) for s in range(3))

    h = 1e-6
    g = synth.rng(1)
    for _ in range(4):
        i, j = (int(x) for x in g.integers(0, c["K"], 2))
        a1, a2 = lA.copy(), lA.copy()
        a1[i, j] += h
        a2[i, j] -= h
        fd = (total(a1, lB) - total(a2, lB)) / (2 * h)
        assert abs(gA[i, j] - fd) <= 1e-4 * abs(fd) + 2e-5
    for _ in range(3):
        j, k = int(g.integers(0, c["K"])), int(g.integers(0, c["M"]))
        b1, b2 = lB.copy(), lB.copy()
        b1[j, k] += h
        b2[j, k] -= h
        fd = (total(lA, b1) - total(lA, b2)) / (2 * h)
        assert abs(gB[j, k] - fd) <= 1e-4 * abs(fd) + 2e-5


def test_autograd_function():
    p = synth.hmm_workload(4, 16, 6, 11, "uniform", 5, 80)
    logs, t, obs, off = _dev(p)
    lA = t["log_A"].clone().requires_grad_(True)
    lB = t["log_B"].clone().requires_grad_(True)
    lpi = t["log_pi"].clone().requires_grad_(True)
    ll = api.HMMLogLik.apply(lA, lB, lpi, obs, off)
    w = torch.linspace(0.5, 1.5, 11, dtype=torch.float64, device=DEV)
    (ll * w).sum().backward()
    _, rA, rB, rpi = ohmm.gradients_batch(p, weights=w.cpu().numpy(), params=ohmm.params_from_f32_logs(logs))
    _check_grads((lA.grad.cpu().numpy(), lB.grad.cpu().numpy(), lpi.grad.cpu().numpy()), (rA, rB, rpi))


def test_single_step_sequences_and_debug_max_T():
    p = synth.hmm_workload(2, 8, 4, 10, "uniform", 1, 3)
    logs, t, obs, off = _dev(p)
    gA, gB, gpi, _ = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    _, rA, rB, rpi = ohmm.gradients_batch(p, params=ohmm.params_from_f32_logs(logs))
    np.testing.assert_allclose(gB.cpu().numpy(), rB, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(gpi.cpu().numpy(), rpi, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(gA.cpu().numpy(), rA, rtol=1e-5, atol=1e-6)
    api.set_debug(True)
    try:
        with pytest.raises(_lib.AccelError) as e:
            api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=1)
        assert e.value.status == 2
    finally:
        api.set_debug(False)


# ------------------------------------------------- forward -> adjoint hand-off (saved state)
@pytest.mark.parametrize("K,M,S,lo,hi", [(256, 64, 24, 200, 2000), (37, 11, 13, 1, 130), (64, 8, 200, 5, 60)])
def test_split_forward_backward_equals_one_call(K, M, S, lo, hi):
    # hmm_adjoint_forward + hmm_adjoint_backward compute exactly what hmm_adjoint does (the same
    # kernels in the same order), and one saved state serves two backward calls with other weights
    p = synth.hmm_workload(K + 2 * S, K, M, S, "uniform", lo, hi)
    logs, t, obs, off = _dev(p)
    ll, saved = api.hmm_adjoint_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    for seed in (1, 2):
        w = torch.from_numpy(synth.rng(seed).uniform(0.0, 2.0, size=S)).to(DEV)
        g2 = api.hmm_adjoint_backward(t["log_A"], t["log_B"], t["log_pi"], obs, off, saved, weights=w)
        g1 = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w)
        for a, b in zip(g2, g1[:3]):
            assert torch.equal(a, b)
        assert torch.equal(ll, g1[3])


def test_autograd_fp32_uses_one_forward_pass():
    # with FP32 precision the autograd forward is the adjoint's checkpointed forward: its logL
    # matches the log-space kernel and the oracle, and the backward matches the oracle
    p = synth.hmm_workload(9, 64, 16, 30, "uniform", 20, 300)
    logs, t, obs, off = _dev(p)
    lA = t["log_A"].clone().requires_grad_(True)
    ll = api.HMMLogLik.apply(lA, t["log_B"], t["log_pi"], obs, off)
    ref_ll = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    assert torch.max(torch.abs(ll.detach() - ref_ll) / torch.abs(ref_ll)).item() <= 1e-5
    ll.sum().backward()
    _, rA, _, _ = ohmm.gradients_batch(p, params=ohmm.params_from_f32_logs(logs))
    np.testing.assert_allclose(lA.grad.cpu().numpy(), rA, rtol=1e-4, atol=1e-6 * rA.sum(axis=1, keepdims=True).max())


@pytest.mark.parametrize("K,M,S,lo,hi", [(64, 8, 200, 5, 60), (128, 16, 100, 10, 300)])
def test_repeated_calls_are_bit_identical(K, M, S, lo, hi):
    # many equal lengths (ties in the length sort); the workspace of each call is a fresh
    # allocation whose stale contents differ, so nothing may depend on them or on timing
    p = synth.hmm_workload(K + 3 * S, K, M, S, "uniform", lo, hi)
    logs, t, obs, off = _dev(p)
    w = torch.from_numpy(synth.rng(3).uniform(0.0, 2.0, size=S)).to(DEV)
    ref = None
    for rep in range(4):
        junk = torch.rand(1 << 24, device=DEV) * rep      # changes what stale memory holds
        del junk
        g = [x.clone() for x in api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w)[:4]]
        if ref is None:
            ref = g
        else:
            for a, b in zip(g, ref):
                assert torch.equal(a, b)


@pytest.mark.parametrize("budget", [40, 8])
def test_sm_budget_gives_identical_results(budget):
    # the forward recursion on fewer SMs (more groups per CTA pair) computes every sequence
    # with the same arithmetic: logL, checkpoints and gradients are bit-identical
    p = synth.hmm_workload(77, 256, 64, 200, "uniform", 50, 500)
    logs, t, obs, off = _dev(p)
    w = torch.from_numpy(synth.rng(7).uniform(0.0, 2.0, size=200)).to(DEV)
    ref = [x.clone() for x in api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w)[:4]]
    try:
        api.set_sm_budget(budget)
        assert api.get_sm_budget() == budget
        got = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w)[:4]
        ll, saved = api.hmm_adjoint_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    finally:
        api.set_sm_budget(0)
    g2 = api.hmm_adjoint_backward(t["log_A"], t["log_B"], t["log_pi"], obs, off, saved, weights=w)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    for a, b in zip(g2, ref[:3]):
        assert torch.equal(a, b)
    assert torch.equal(ll, ref[3])


@pytest.mark.parametrize("K,M,S,lo,hi", [(64, 8, 200, 5, 60), (256, 64, 40, 50, 300)])
def test_adjoint_captured_in_a_cuda_graph_replays_bit_identical(K, M, S, lo, hi):
    # the backward phase forks to its own two streams and joins the caller's stream again with
    # events, so a whole call captures into a CUDA graph; replays give the eager results
    p = synth.hmm_workload(K + 5 * S, K, M, S, "uniform", lo, hi)
    logs, t, obs, off = _dev(p)
    max_T = int(p["lengths"].max())
    w = torch.from_numpy(synth.rng(9).uniform(0.5, 2.0, size=S)).to(DEV)
    ref = [x.clone() for x in api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w,
                                              max_T=max_T)[:4]]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                      # warm-up on a non-default stream
        api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w, max_T=max_T)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w, max_T=max_T)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(out[:4], ref):
            assert torch.equal(a, b)


def test_adjoint_orders_with_the_callers_stream():
    # on a side stream: a long kernel, then the weights written, then the call, then the
    # gradients read -- all enqueued back to back with no host synchronisation.  The backward's
    # own streams fork from the caller's stream after the weights are written and join it
    # before the gradients are read, so the results equal a call on settled inputs.
    K, M, S = 128, 16, 120
    p = synth.hmm_workload(606, K, M, S, "uniform", 20, 200)
    logs, t, obs, off = _dev(p)
    max_T = int(p["lengths"].max())
    w_host = synth.rng(12).uniform(0.5, 2.0, size=S)
    w_ref = torch.from_numpy(w_host).to(DEV)
    ref = [x.clone() for x in api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w_ref,
                                              max_T=max_T)[:3]]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    big = torch.randn(4096, 4096, device=DEV)
    w = torch.zeros(S, dtype=torch.float64, device=DEV)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(4):
            big = big @ big / 64.0                     # keeps the stream busy for a while
        w.copy_(w_ref)
        g = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, weights=w, max_T=max_T)[:3]
        got = [x.clone() for x in g]
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_adjoint_from_two_host_threads_at_once():
    # each host thread gets the backward's streams of its own; two calls in flight at once
    # on two streams give the results of the same calls one after the other
    import threading
    cases = []
    for seed, (K, M, S) in enumerate([(64, 8, 150), (256, 64, 30)]):
        p = synth.hmm_workload(700 + seed, K, M, S, "uniform", 30, 250)
        logs, t, obs, off = _dev(p)
        cases.append((t, obs, off, int(p["lengths"].max())))
    ref = []
    for t, obs, off, mt in cases:
        ref.append([x.clone() for x in api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=mt)[:4]])
    torch.cuda.synchronize()
    out = [None, None]
    errs = []

    def run(i):
        try:
            t, obs, off, mt = cases[i]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(3):
                    g = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=mt)[:4]
                out[i] = [x.clone() for x in g]
            s.synchronize()
        except Exception as e:                      # surfaced below
            errs.append(e)

    th = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errs, errs
    for got, r in zip(out, ref):
        for a, b in zip(got, r):
            assert torch.equal(a, b)
