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
