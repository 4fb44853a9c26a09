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


# ---------------------------------------------------------------------------------------
# The batched configuration (K=256, M=64, 4,096 sequences, lengths log-uniform in [50, 5000])
# compared on EVERY sequence.  The float64 oracle is evaluated three ways (once each, shared
# by the tests below): on the float32-rounded log parameters the library receives (the
# parity reading); on the original float64 parameters (the total error, parameter rounding
# included); and on the parameters as the kernel holds them, A and B rounded to bfloat16 (the
# error of the BF16 arithmetic alone: the alpha tile rounded to BF16 every step).
_FULL = {}


def _batched_full():
    if not _FULL:
        c = synth.CFG_HMM_BATCHED
        p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
        logs = synth.hmm_log_inputs_f32(p)
        _FULL["p"] = p
        _FULL["fp32_params"] = ohmm.loglik_scaled_batch(p, params=ohmm.params_from_f32_logs(logs))
        _FULL["original"] = ohmm.loglik_scaled_batch(p)
        _FULL["bf16_params"] = ohmm.loglik_scaled_batch(p, params=ohmm.params_bf16_from_f32_logs(logs))
    return _FULL


def _rel(ll, ref):
    return np.abs(ll - ref) / np.abs(ref)


def _full_bf16_run(tmp_path=None, force=None):
    f = _batched_full()
    p = f["p"]
    logs, t, obs, off = _prep(p)
    if force is not None:
        t["obs"], t["off"] = obs, off
        _force_config(tmp_path, p["K"], p["M"], p["S"], *force[:2], t, pair=force[2])
    else:
        api.hmm_autotune(t["log_A"], t["log_B"], t["log_pi"], obs, off)     # the bench's choice
    ll = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED).cpu().numpy()
    assert np.all(np.isfinite(ll))
    return f, ll


def _report(tag, rel):
    print(f"\n[bf16 logL error, {tag}] max {rel.max():.3e}  p99 {np.percentile(rel, 99):.3e}  "
          f"median {np.median(rel):.3e}  over {rel.size} sequences")


def test_bf16_tc_config_all_sequences_autotuned():
    f, ll = _full_bf16_run()
    for tag in ("fp32_params", "original", "bf16_params"):
        rel = _rel(ll, f[tag])
        _report(tag, rel)
        assert rel.max() <= 1e-3, (tag, rel.max())


@pytest.mark.parametrize("split,rows,pair", [(2, 128, 0), (4, 64, 1), (4, 32, 1), (2, 64, 2), (2, 32, 2)])
def test_bf16_tc_config_all_sequences_each_launch_shape(tmp_path, split, rows, pair):
    f, ll = _full_bf16_run(tmp_path, (split, rows, pair))
    rel = _rel(ll, f["fp32_params"])
    _report(f"fp32_params, split={split} rows={rows} pair={pair}", rel)
    assert rel.max() <= 1e-3


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


def _force_config(tmp_path, K, M, S, split, rows, t, pair=0, units=None):
    import json as _json
    path = str(tmp_path / "tune.jsonl")
    sl = 0
    while (1 << (sl + 1)) <= S:
        sl += 1
    entry = {"kernel": "hmm_forward_bf16", "device": torch.cuda.get_device_name(), "K": K, "M": M,
             "S_log2": sl, "split": split, "rows": rows, "pair": pair}
    if units is not None:                  # lines without "units" launch all units
        entry["units"] = units
    entry["ms"] = 1.0
    with open(path, "w") as f:
        f.write(_json.dumps(entry) + "\n")
    ms, cfg = api.hmm_autotune(t["log_A"], t["log_B"], t["log_pi"], t["obs"], t["off"], cache_path=path)
    assert ms == 0.0 and cfg == (split, rows, pair, units or 0)


@pytest.mark.parametrize("split,rows", [(2, 128), (4, 128), (4, 32), (2, 64), (4, 64), (2, 32)])
def test_bf16_tc_launch_configurations(tmp_path, split, rows):
    p = synth.hmm_workload(12, 128, 32, 700, "loguniform", 1, 400)
    logs, t, obs, off = _prep(p)
    t["obs"], t["off"] = obs, off
    _force_config(tmp_path, 128, 32, 700, split, rows, t)
    _check(p, acc.HMM_BF16_SCALED)


# cluster pair (two CTAs split the state columns): K=128 runs 2 parts of 32 columns per
# CTA, K=256 2 or 4 parts; 700 sequences over 32-row tiles also exercise the one-step hand-off
# of queue indices from the first CTA of a pair to the second
@pytest.mark.parametrize("K,split,rows", [(128, 2, 128), (128, 2, 32), (256, 4, 64), (256, 2, 128), (256, 4, 32)])
def test_bf16_tc_cluster_pair(tmp_path, K, split, rows):
    p = synth.hmm_workload(14, K, 40, 700, "loguniform", 1, 400)
    logs, t, obs, off = _prep(p)
    t["obs"], t["off"] = obs, off
    _force_config(tmp_path, K, 40, 700, split, rows, t, pair=1)
    _check(p, acc.HMM_BF16_SCALED)


# clusters of four CTAs (K/4 = 64 state columns each, MMA N = 64): CTA 0 pops the queue and
# mails the index to the other three; rows of 128, 64 and 32
@pytest.mark.parametrize("rows", [128, 64, 32])
def test_bf16_tc_cluster_of_four(tmp_path, rows):
    p = synth.hmm_workload(15, 256, 40, 700, "loguniform", 1, 400)
    logs, t, obs, off = _prep(p)
    t["obs"], t["off"] = obs, off
    _force_config(tmp_path, 256, 40, 700, 2, rows, t, pair=2)
    _check(p, acc.HMM_BF16_SCALED)


def test_autotune_times_candidates_and_caches(tmp_path):
    c = synth.CFG_HMM_BATCHED
    p = synth.hmm_workload(c["seed"], c["K"], c["M"], 512, c["kind"], c["lo"], 600)
    logs, t, obs, off = _prep(p)
    path = str(tmp_path / "tune.jsonl")
    ms, cfg = api.hmm_autotune(t["log_A"], t["log_B"], t["log_pi"], obs, off, cache_path=path)
    assert ms > 0.0 and cfg[0] in (2, 4) and cfg[1] in (32, 64, 128) and cfg[2] in (0, 1, 2) and cfg[3] >= 0
    with open(path) as f:
        assert "hmm_forward_bf16" in f.read()
    ms2, cfg2 = api.hmm_autotune(t["log_A"], t["log_B"], t["log_pi"], obs, off, cache_path=path)
    assert ms2 == 0.0 and cfg2 == cfg                      # taken from the cache file
    _check(p, acc.HMM_BF16_SCALED, sample=list(range(0, 512, 37)))


def test_graph_capture_replays_the_persistent_launch():
    p = synth.hmm_workload(13, 256, 64, 600, "loguniform", 50, 800)
    logs, t, obs, off = _prep(p)
    direct = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED)
    from paper_2211_00621_gb300 import _lib
    import ctypes as C
    lib = _lib.load()
    m = api._model(t["log_A"], t["log_B"], t["log_pi"])
    ws = torch.empty(lib.hmm_forward_workspace_size(C.byref(m), 600, obs.numel(), acc.HMM_BF16_SCALED),
                     dtype=torch.uint8, device=DEV)
    out = torch.full((600,), float("nan"), dtype=torch.float64, device=DEV)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = api.Graph()
    g.capture(lambda: api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED,
                                      out=out, ws=ws), stream=side)
    assert g.nodes() >= 2
    for _ in range(2):
        out.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(out, direct)


# fewer persistent work units than fit (the autotuner's choice for a latency-bound mix): the
# queue hands every tile to one of the launched CTAs / clusters all the same
@pytest.mark.parametrize("pair,units", [(0, 1), (0, 5), (1, 1), (1, 3), (2, 2)])
def test_bf16_tc_fewer_work_units(tmp_path, pair, units):
    p = synth.hmm_workload(16, 256, 40, 700, "loguniform", 1, 400)
    logs, t, obs, off = _prep(p)
    t["obs"], t["off"] = obs, off
    _force_config(tmp_path, 256, 40, 700, 2, 64, t, pair=pair, units=units)
    _check(p, acc.HMM_BF16_SCALED)
