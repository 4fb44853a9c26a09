"""Parity of the re-estimation step (softmax-parameterised gradient and Baum-Welch M-step)
against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import hmm as ohmm
from paper_2211_00621_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _inputs(seed, K, M, zero_rows=()):
    p = synth.hmm_workload(seed, K, M, 2, "fixed", 3, 3)     # the parameters only
    logs = synth.hmm_log_inputs_f32(p)
    rng = np.random.default_rng(seed + 1000)
    g = {"A": rng.gamma(0.7, 3.0, size=(K, K)), "B": rng.gamma(0.7, 3.0, size=(K, M)), "pi": rng.gamma(0.7, 3.0, size=K)}
    g = {k: v.astype(np.float32) for k, v in g.items()}
    for r in zero_rows:
        g["A"][r] = 0.0
        g["B"][r] = 0.0
        g["B"][(r + 1) % K, : M // 2] = 0.0                 # zero counts inside a row with a positive sum
    return logs, g


def _run(logs, g):
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    gd = [torch.from_numpy(g[k]).to(DEV) for k in ("A", "B", "pi")]
    th, nw = api.hmm_mstep(t["log_A"], t["log_B"], t["log_pi"], *gd)
    return [x.cpu().numpy() for x in th], [x.cpu().numpy() for x in nw]


def _check(logs, g, th, nw):
    for i, (name, lk) in enumerate((("A", "log_A"), ("B", "log_B"), ("pi", "log_pi"))):
        logP = logs[lk].astype(np.float64)
        gg = g[name].astype(np.float64)
        ref_t = ohmm.softmax_rows_grad(logP, gg)
        ref_n = ohmm.mstep_rows(gg, logP)
        # theta gradient g - P sum(g): P from expf of an FP32 difference log P - max (relative
        # error up to (|log P - max| + 4) 2^-24, under 1e-6 for the rows here), sums in FP64, one
        # FP32 rounding of the result
        P = np.exp(logP - ohmm._lse(logP, axis=-1)[..., None])
        scale = np.abs(gg) + P * np.abs(gg.sum(axis=-1, keepdims=True))
        assert np.all(np.abs(th[i] - ref_t) <= 2e-6 * scale + 1e-30), name
        # new log parameters: equal infinities, else within logf's few-ulp error plus one FP32
        # rounding of log values
        fin = np.isfinite(ref_n)
        assert np.array_equal(np.isinf(nw[i]), ~fin), name
        np.testing.assert_allclose(nw[i][fin], ref_n[fin], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("K,M", [(1, 1), (1, 7), (7, 5), (64, 64), (256, 64), (256, 300), (200, 1024)])
def test_mstep_matches_oracle(K, M):
    logs, g = _inputs(K * 7 + M, K, M)
    th, nw = _run(logs, g)
    _check(logs, g, th, nw)


def test_mstep_zero_count_rows_keep_parameters():
    logs, g = _inputs(42, 64, 32, zero_rows=(3, 17))
    th, nw = _run(logs, g)
    _check(logs, g, th, nw)
    np.testing.assert_array_equal(nw[0][3], logs["log_A"][3])
    np.testing.assert_array_equal(nw[1][17], logs["log_B"][17])


def test_mstep_outputs_may_be_skipped():
    logs, g = _inputs(9, 32, 16)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    gd = [torch.from_numpy(g[k]).to(DEV) for k in ("A", "B", "pi")]
    th, nw = api.hmm_mstep(t["log_A"], t["log_B"], t["log_pi"], *gd, want_grad=False)
    assert th is None and len(nw) == 3
    th2, nw2 = api.hmm_mstep(t["log_A"], t["log_B"], t["log_pi"], *gd, want_new=False)
    assert nw2 is None
    _check(logs, g, [x.cpu().numpy() for x in th2], [x.cpu().numpy() for x in nw])


def test_adjoint_then_mstep_is_one_baum_welch_iteration():
    # counts from the GPU adjoint, re-estimated on the GPU, against the oracle's own counts
    p = synth.hmm_workload(21, 16, 8, 40, "uniform", 5, 60)
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    obs = torch.from_numpy(p["obs"]).to(DEV)
    off = torch.from_numpy(p["offsets"]).to(DEV)
    gA, gB, gpi, _ = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    _, nw = api.hmm_mstep(t["log_A"], t["log_B"], t["log_pi"], gA, gB, gpi, want_grad=False)
    q = ohmm.params_from_f32_logs(logs)
    _, rA, rB, rpi = ohmm.gradients_batch(p, params=q)
    for got, g, lk in zip(nw, (rA, rB, rpi), ("log_A", "log_B", "log_pi")):
        ref = ohmm.mstep_rows(g, logs[lk].astype(np.float64))
        np.testing.assert_allclose(got.cpu().numpy(), ref, atol=1e-3)
    # the re-estimated model does not lower the likelihood (EM)
    new = {k: np.exp(v.cpu().numpy().astype(np.float64)) for k, v in zip(("A", "B", "pi"), nw)}
    assert ohmm.loglik_batch(p, params=new).sum() >= ohmm.loglik_batch(p, params=q).sum() - 1e-3
