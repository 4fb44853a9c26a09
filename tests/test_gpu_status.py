"""Debug mode and error statuses of the C ABI (the paper's debug-mode runtime checks,
Sec. 3.2 and Appendix B): every invalid input is rejected with its status code and no
GPU fault."""
import numpy as np
import pytest
import torch

import paper_2211_00621_gb300 as acc
from paper_2211_00621_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture
def debug():
    api.set_debug(True)
    yield
    api.set_debug(False)


def _status(fn, *a, **k):
    with pytest.raises(_lib.AccelError) as e:
        fn(*a, **k)
    return e.value.status


def test_bad_offsets_rejected_in_debug_mode(debug):
    data = torch.arange(100, dtype=torch.int32, device=DEV)
    off = torch.tensor([0, 50, 40, 100], dtype=torch.int64, device=DEV)      # not monotone
    assert _status(api.accel_segreduce, acc.RED_ADD, acc.MAP_IDENTITY, data, off) == 2
    off = torch.tensor([0, 50, 60, 99], dtype=torch.int64, device=DEV)       # offsets[S] != N
    assert _status(api.accel_segreduce, acc.RED_ADD, acc.MAP_IDENTITY, data, off) == 2


def test_symbol_out_of_range_rejected_in_debug_mode(debug):
    p = synth.hmm_workload(0, 8, 4, 3, "fixed", 10, 10)
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    obs = torch.from_numpy(p["obs"]).to(DEV)
    obs[5] = 4
    off = torch.from_numpy(p["offsets"]).to(DEV)
    assert _status(api.hmm_forward, t["log_A"], t["log_B"], t["log_pi"], obs, off) == 2
    obs[5] = 0
    off0 = off.clone()
    off0[1] = off0[0]                                                          # empty sequence
    assert _status(api.hmm_forward, t["log_A"], t["log_B"], t["log_pi"], obs, off0) == 2
    api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off)            # valid input passes


def test_bad_arguments():
    x = torch.zeros(10, dtype=torch.int32, device=DEV)
    assert _status(api.accel_map, 99, x) == 1
    assert _status(api.accel_map, acc.MAP_SQ_PLUS_ONE, x.float(), torch.int64) == 3   # float -> int
    t4 = torch.zeros(2, 2, 2, 2, dtype=torch.float32, device=DEV)
    assert _status(api.accel_loop, acc.LOOP_SCALE, t4, t4, 2.0) == 2          # rank 4 > 3
    assert _status(api.accel_loop, acc.LOOP_SCALE, x, x.float(), 2.0) == 3


def test_unsupported_hmm_shape():
    K, M = 300, 4
    lA = torch.zeros(K, K, device=DEV)
    lB = torch.zeros(K, M, device=DEV)
    lpi = torch.zeros(K, device=DEV)
    obs = torch.zeros(4, dtype=torch.int32, device=DEV)
    off = torch.tensor([0, 4], dtype=torch.int64, device=DEV)
    assert _status(api.hmm_forward, lA, lB, lpi, obs, off) == 7


def test_workspace_too_small_for_segreduce():
    lib = _lib.load()
    x = torch.zeros(10, dtype=torch.int32, device=DEV)
    off = torch.tensor([0, 10], dtype=torch.int64, device=DEV)
    out = torch.empty(1, dtype=torch.int64, device=DEV)
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    need = lib.accel_segreduce_workspace_size(10, 1)
    st = lib.accel_segreduce(acc.RED_ADD, acc.MAP_IDENTITY, acc.I32, acc.I64, x.data_ptr(), 10, off.data_ptr(), 1,
                             0.0, out.data_ptr(), ws.data_ptr(), need - 1, None)
    assert st == 4
    assert b"workspace" in lib.accel_last_error()


# ------------------------------------------------- device status word in accelerate mode
@pytest.fixture
def status_word():
    word = torch.zeros(1, dtype=torch.int32, device=DEV)
    api.set_device_status(word)
    yield word
    api.set_device_status(None)


def _hmm_dev(p):
    logs = synth.hmm_log_inputs_f32(p)
    t = {k: torch.from_numpy(v).to(DEV) for k, v in logs.items()}
    return logs, t, torch.from_numpy(p["obs"]).to(DEV), torch.from_numpy(p["offsets"]).to(DEV)


# K = 64 takes the cluster-pair adjoint kernels, K = 37 the streaming ones
@pytest.mark.parametrize("K,M", [(64, 8), (37, 5)])
def test_adjoint_max_T_too_small_reported_in_accelerate_mode(status_word, K, M):
    from oracle import hmm as ohmm
    p = synth.hmm_workload(21 + K, K, M, 40, "uniform", 20, 60)
    logs, t, obs, off = _hmm_dev(p)
    assert not _lib.load().accel_get_debug()
    # max_T = 4 sizes checkpoint segments of 2 steps: every sequence (>= 20 steps) is too long;
    # the call itself returns OK (accelerate mode) and the error waits in the status word
    api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=4)
    with pytest.raises(_lib.AccelError) as e:
        api.sync_status(status_word)
    assert e.value.status == 2 and "max_T" in str(e.value)
    assert int(status_word.item()) == 0                      # cleared by sync_status
    # a correctly sized call leaves the word at OK and matches the oracle
    gA, gB, gpi, _ = api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)
    api.sync_status(status_word)
    _, rA, rB, rpi = ohmm.gradients_batch(p, params=ohmm.params_from_f32_logs(logs))
    for g, r in ((gA, rA), (gB, rB), (gpi, rpi)):
        assert np.linalg.norm(g.cpu().numpy() - r) <= 1e-4 * np.linalg.norm(r)


def test_first_error_stays_until_cleared(status_word):
    p = synth.hmm_workload(23, 64, 8, 12, "uniform", 30, 50)
    _, t, obs, off = _hmm_dev(p)
    api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off, max_T=4)    # SHAPE
    api.hmm_adjoint(t["log_A"], t["log_B"], t["log_pi"], obs, off)             # fine: does not clear
    with pytest.raises(_lib.AccelError) as e:
        api.sync_status(status_word, clear=False)
    assert e.value.status == 2
    assert int(status_word.item()) == 2                      # kept (clear=False)
    status_word.zero_()
    api.sync_status(status_word)


def _force_single_cta(tmp_path, K, M, S, t, obs, off, split=2, rows=64):
    import json
    path = str(tmp_path / "tune.jsonl")
    sl = S.bit_length() - 1
    with open(path, "w") as f:
        f.write(json.dumps({"kernel": "hmm_forward_bf16", "device": torch.cuda.get_device_name(), "K": K, "M": M,
                            "S_log2": sl, "split": split, "rows": rows, "pair": 0, "ms": 1.0}) + "\n")
    ms, cfg = api.hmm_autotune(t["log_A"], t["log_B"], t["log_pi"], obs, off, cache_path=path)
    assert ms == 0.0 and cfg == (split, rows, 0, 0)


def test_watchdog_stops_single_cta_bf16_forward_with_timeout(status_word, tmp_path):
    # The persistent single-CTA BF16 forward with a 1 us run-time budget stops at its next step
    # boundary (its tensor-core work of the previous step complete), frees its tensor memory and
    # reports TIMEOUT; the context stays usable and the next call, without a budget, is correct.
    from oracle import hmm as ohmm
    K, M, S = 128, 32, 700
    p = synth.hmm_workload(31, K, M, S, "loguniform", 50, 400)
    logs, t, obs, off = _hmm_dev(p)
    _force_single_cta(tmp_path, K, M, S, t, obs, off)
    try:
        api.set_watchdog_ns(1000)
        api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED)
        with pytest.raises(_lib.AccelError) as e:
            api.sync_status(status_word)
        assert e.value.status == 6
    finally:
        api.set_watchdog_ns(0)
    ll = api.hmm_forward(t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED)
    api.sync_status(status_word)
    ref = ohmm.loglik_batch(p, seqs=range(0, S, 50), params=ohmm.params_from_f32_logs(logs))
    got = ll.cpu().numpy()[::50]
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-3


def test_watchdog_timeout_in_debug_mode_is_returned(tmp_path):
    K, M, S = 128, 32, 700
    p = synth.hmm_workload(31, K, M, S, "loguniform", 50, 400)
    _, t, obs, off = _hmm_dev(p)
    _force_single_cta(tmp_path, K, M, S, t, obs, off)
    api.set_debug(True)
    api.set_watchdog_ns(1000)
    try:
        assert _status(api.hmm_forward, t["log_A"], t["log_B"], t["log_pi"], obs, off, acc.HMM_BF16_SCALED) == 6
    finally:
        api.set_watchdog_ns(0)
        api.set_debug(False)


@pytest.mark.parametrize("S", [0, 1, 5, 4096, 100_000])
def test_hmm_max_length(S):
    lengths = synth.seq_lengths(3, S, "loguniform", 1, 5000)
    off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    got = int(api.hmm_max_length(torch.from_numpy(off).to(DEV)).item())
    assert got == (int(lengths.max()) if S else 0)
