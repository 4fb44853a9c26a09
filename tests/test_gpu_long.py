"""Parity of the parallel-in-T forward (chunked products of A diag(b(o_t))) with the oracle's
sequential forward, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import hmm as ohmm
from paper_2211_00621_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
# FP32 products: each step rounds every entry (a 64-term sum) once; the error of logL grows
# like the square root of the number of steps, far below 1e-6 of |logL| at these lengths
TOL = 1e-6


def _prep(p):
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    return logs, t, torch.from_numpy(p["obs"]).to(DEV), torch.from_numpy(p["offsets"]).to(DEV)


def _check(p, seqs=None, max_T=None):
    logs, t, obs, off = _prep(p)
    ll = api.hmm_forward_long(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=max_T).cpu().numpy()
    idx = np.arange(p["S"]) if seqs is None else np.asarray(seqs)
    ref = ohmm.loglik_batch(p, seqs=idx, params=ohmm.params_from_f32_logs(logs))
    assert np.all(np.isfinite(ll))
    rel = np.abs(ll[idx] - ref) / np.abs(ref)
    assert rel.max() <= TOL, f"max rel err {rel.max():.3e}"
    return ll


@pytest.mark.parametrize("K,M", [(1, 3), (5, 7), (32, 300), (64, 64)])
def test_long_matches_oracle_mixed_lengths(K, M):
    # lengths 1 and 2 (no or one matrix), shorter than the chunk count, and long
    p = synth.hmm_workload(K * 3 + M, K, M, 9, "uniform", 1, 3000)
    lens = np.array([1, 2, 3, 17, 64, 65, 1500, 2999, 3000])
    p["lengths"] = lens
    p["offsets"] = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    rng = np.random.default_rng(K + M)
    p["obs"] = rng.integers(0, M, size=int(lens.sum())).astype(np.int32)
    _check(p)


def test_long_single_sequence_many_chunks():
    p = synth.hmm_workload(31, 48, 20, 1, "fixed", 40000, 40000)
    _check(p)


def test_long_max_T_above_the_longest_sequence():
    p = synth.hmm_workload(32, 16, 8, 5, "uniform", 100, 900)
    _check(p, max_T=5000)


def test_long_agrees_with_the_fp32_log_forward():
    p = synth.hmm_workload(33, 64, 32, 6, "uniform", 500, 4000)
    logs, t, obs, off = _prep(p)
    a = api.hmm_forward_long(t["log_A"], t["log_B"], t["log_pi"], obs, off).cpu().numpy()
    b = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, api.HMM_FP32_LOG).cpu().numpy()
    assert (np.abs(a - b) / np.abs(b)).max() <= 2e-6


def test_long_bench_config_all_sequences():
    c = synth.CFG_HMM_LONG
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
    _check(p)


def test_long_rejects_k_above_64():
    from paper_2211_00621_gb300 import _lib
    p = synth.hmm_workload(1, 65, 4, 2, "fixed", 5, 5)
    logs, t, obs, off = _prep(p)
    with pytest.raises(_lib.AccelError) as e:
        api.hmm_forward_long(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    assert e.value.status == 7
