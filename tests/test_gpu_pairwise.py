"""GPU parity of the all-pairs map-of-reduce with the float64 oracle, through the C ABI.

Criterion per body: |a_gpu - a_ref| <= 1e-4 * max(|a_ref|, sum_j |term_ij| / sqrt(N)), i.e.
relative 1e-4 except where the net force cancels, where the scale of the summed terms
(which sets the FP32 rounding error of the sum) is used instead.
"""
import numpy as np
import pytest
import torch

from paper_2211_00621_gb300 import api, synth
from oracle import pairwise as opair

pytestmark = pytest.mark.gpu
DEV = "cuda"
F32 = torch.float32


def _run(b, eps):
    aos = torch.from_numpy(b["aos"]).to(DEV)
    x, y, z, m = api.accel_marshal_records(aos, [(0, F32), (4, F32), (8, F32), (12, F32)])
    ax, ay, az = api.pairwise_mapreduce(x, y, z, m, eps)
    return torch.stack([ax, ay, az], 1).cpu().numpy().astype(np.float64)


def _check(b, eps, idx):
    a = _run(b, eps)
    pos, mass = b["aos"][:, :3], b["aos"][:, 3]
    ref = opair.accel(pos, mass, eps, idx)
    scale = np.maximum(np.linalg.norm(ref, axis=1), opair.term_scale(pos, mass, eps, idx))
    err = np.linalg.norm(a[idx] - ref, axis=1)
    assert np.all(err <= 1e-4 * scale), f"max scaled err {np.max(err / scale):.3e}"
    return a


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 511, 512, 513, 1000, 1025, 3000, 4099, 9001])
def test_small_all_bodies(n):
    # n < 2,048 runs one CTA per 64 bodies; 3,000, 4,099 and 9,001 split the j range over
    # clusters of 2, 4 and 8 CTAs
    b = synth.bodies(n, n)
    _check(b, 1e-3, list(range(n)))


def test_config_sampled_and_zero_net_momentum():
    c = synth.CFG_ALLPAIRS
    b = synth.bodies(c["seed"], c["N"])
    idx = list(range(0, c["N"], 1021)) + [c["N"] - 1]
    a = _check(b, c["eps"], idx)
    m = b["aos"][:, 3].astype(np.float64)
    net = (m[:, None] * a).sum(axis=0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.abs(net).max() <= 1e-5 * scale


def test_two_body_closed_form():
    aos = np.array([[0.1, 0.2, 0.3, 2.0], [0.4, -0.2, 0.3, 3.0]], dtype=np.float32)
    a = _run({"aos": aos}, 1e-3)
    d = aos[1, :3].astype(np.float64) - aos[0, :3]
    r2 = float(d @ d) + 1e-6
    np.testing.assert_allclose(a[0], 3.0 * d / r2 ** 1.5, rtol=2e-6)
    np.testing.assert_allclose(a[1], -2.0 * d / r2 ** 1.5, rtol=2e-6)


@pytest.mark.parametrize("eps", [0.0, -1e-3, float("nan"), float("inf"), 1e-14])
def test_eps_outside_its_range_is_rejected(eps):
    # eps^-3 must be finite in FP32 (the j = i term is 0 * m_i eps^-3); nothing is launched
    b = synth.bodies(0, 8)
    with pytest.raises(RuntimeError, match="eps"):
        _run(b, eps)


def test_ragged_pointer_offsets():
    # inputs that start at an element offset (not 16-byte aligned): the j tiles are loaded
    # element by element, so any float alignment is accepted
    b = synth.bodies(5, 1001)
    aos = torch.from_numpy(b["aos"]).to(DEV)
    x, y, z, m = api.accel_marshal_records(aos, [(0, F32), (4, F32), (8, F32), (12, F32)])
    sub = [v[1:] for v in (x, y, z, m)]
    ax, ay, az = api.pairwise_mapreduce(*sub, 1e-3)
    a = torch.stack([ax, ay, az], 1).cpu().numpy().astype(np.float64)
    pos, mass = b["aos"][1:, :3], b["aos"][1:, 3]
    idx = list(range(1000))
    ref = opair.accel(pos, mass, 1e-3, idx)
    scale = np.maximum(np.linalg.norm(ref, axis=1), opair.term_scale(pos, mass, 1e-3, idx))
    assert np.all(np.linalg.norm(a - ref, axis=1) <= 1e-4 * scale)
