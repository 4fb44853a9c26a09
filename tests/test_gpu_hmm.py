"""GPU parity of the HMM forward kernels with the float64 oracle, through the C ABI.

Tolerances (relative, per sequence, on logL): 1e-5 for the FP32 log-space kernel and
1e-3 for the BF16 tensor-core kernel, against the oracle evaluated on the same
float32-rounded log parameters the kernels receive.
"""
import numpy as np
import pytest
import torch

import paper_2211_00621_gb300 as acc
from paper_2211_00621_gb300 import api, synth
from oracle import hmm as ohmm

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = {acc.HMM_FP32_LOG: 1e-5, acc.HMM_BF16_SCALED: 1e-3}


def _prep(p):
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    return logs, t, torch.from_numpy(p["obs"]).to(DEV), torch.from_numpy(p["offsets"]).to(DEV)


def _check(p, precision, sample=None):
    logs, t, obs, off = _prep(p)
    ll = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, precision).cpu().numpy()
    idx = np.arange(p["S"]) if sample is None else np.asarray(sample)
    ref = ohmm.loglik_batch(p, seqs=idx, params=ohmm.params_from_f32_logs(logs))
    rel = np.abs(ll[idx] - ref) / np.abs(ref)
    assert np.all(np.isfinite(ll)), "non-finite logL"
    assert rel.max() <= TOL[precision], f"max rel err {rel.max():.3e}"
    return ll, rel


def test_fp32_plain_config_all_sequences():
    c = synth.CFG_HMM_PLAIN
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
    _check(p, acc.HMM_FP32_LOG)


@pytest.mark.parametrize("K,M", [(1, 3), (5, 7), (32, 16), (48, 40)])
def test_fp32_plain_small_shapes(K, M):
    p = synth.hmm_workload(K + M, K, M, 37, "uniform", 1, 300)
    _check(p, acc.HMM_FP32_LOG)


@pytest.mark.parametrize("K,M", [(96, 20), (256, 64)])
def test_fp32_cta_variant(K, M):
    p = synth.hmm_workload(3, K, M, 45, "loguniform", 1, 400)
    _check(p, acc.HMM_FP32_LOG)


@pytest.mark.parametrize("K,M", [(256, 64), (192, 48), (128, 32), (64, 8)])
def test_bf16_tc_small(K, M):
    p = synth.hmm_workload(5, K, M, 300, "loguniform", 1, 300)
    _check(p, acc.HMM_BF16_SCALED)


def test_bf16_tc_more_sequences_than_rows():
    # more sequences than 148+ CTAs x 128 rows: rows refill from the queue
    p = synth.hmm_workload(6, 64, 16, 160 * 128 + 77, "uniform", 1, 12)
    _check(p, acc.HMM_BF16_SCALED, sample=list(range(0, p["S"], 97)) + [p["S"] - 1])


def test_bf16_tc_config_sampled():
    c = synth.CFG_HMM_BATCHED
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
    L = p["lengths"]
    sample = sorted(set(np.argsort(L)[-6:].tolist() + np.argsort(L)[:4].tolist() + list(range(0, c["S"], 331))))
    _check(p, acc.HMM_BF16_SCALED, sample=sample)


def test_bf16_error_against_original_parameters_reported():
    # total error (rounding of the parameters to FP32 logs and BF16 included) on a sample
    c = synth.CFG_HMM_BATCHED
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], 256, c["kind"], c["lo"], 1000)
    logs, t, obs, off = _prep(p)
    ll = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED).cpu().numpy()
    idx = list(range(0, 256, 16))
    ref = ohmm.loglik_batch(p, seqs=idx)
    assert (np.abs(ll[idx] - ref) / np.abs(ref)).max() <= 1e-3


def test_bf16_tc_rejects_unsupported_k():
    from paper_2211_00621_gb300 import _lib
    p = synth.hmm_workload(1, 32, 8, 4, "fixed", 5, 5)
    logs, t, obs, off = _prep(p)
    with pytest.raises(_lib.AccelError) as e:
        api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED)
    assert e.value.status == 7


def test_single_step_sequences():
    p = synth.hmm_workload(7, 64, 32, 50, "fixed", 1, 1)
    for prec in (acc.HMM_FP32_LOG, acc.HMM_BF16_SCALED):
        _check(p, prec)
