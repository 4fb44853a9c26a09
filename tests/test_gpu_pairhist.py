"""All-pairs angular histogram against the oracle, through the C ABI (bit-exact counts)."""
import numpy as np
import pytest
import torch

from oracle import pairhist as ph
from paper_2211_00621_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
E20 = synth.angle_edges(20, 1.0, 10000.0)


def _gpu(A, e, B=None):
    tb = torch.from_numpy(B).to(DEV) if B is not None else None
    return api.accel_pair_histogram(torch.from_numpy(A).to(DEV), e, tb).cpu().numpy()


@pytest.mark.parametrize("N", [1, 2, 255, 256, 257, 1000, 3000])
def test_self_pairs_match_oracle(N):
    A = synth.sphere_points(N, N)
    assert np.array_equal(_gpu(A, E20), ph.pair_histogram(A, E20))


@pytest.mark.parametrize("NA,NB", [(500, 777), (256, 1), (3, 0), (0, 9)])
def test_cross_pairs_match_oracle(NA, NB):
    A = synth.sphere_points(10 + NA, NA)
    B = synth.sphere_points(20 + NB, NB)
    e = synth.angle_edges(30, 2.0, 6000.0)
    assert np.array_equal(_gpu(A, e, B), ph.pair_histogram(A, e, B))


def test_closed_forms_on_the_gpu():
    k, m = 300, 200
    A = np.array([[0, 0, 1]] * k + [[0, 0, -1]] * m, dtype=np.float32)
    h = _gpu(A, E20)
    assert h[0] == k * (k - 1) // 2 + m * (m - 1) // 2 and h[-1] == k * m and h[1:-1].sum() == 0
    N = 40
    phi = 2 * np.pi * np.arange(N) / N
    P = np.stack([np.cos(phi), np.sin(phi), np.zeros(N)], axis=1).astype(np.float32)
    e = np.cos(np.pi * (2 * np.arange(N // 2) + 1) / N).astype(np.float32)
    expect = np.zeros(N // 2 + 1, dtype=np.int64)
    expect[1:N // 2] = N
    expect[N // 2] = N // 2
    assert np.array_equal(_gpu(P, e), expect)


def test_bench_config_all_pairs():
    c = synth.CFG_PAIRHIST
    A = synth.sphere_points(c["seed"], c["N"])
    e = synth.angle_edges(c["nbins"], c["amin"], c["amax"])
    h = _gpu(A, e)
    assert h.sum() == c["N"] * (c["N"] - 1) // 2
    assert np.array_equal(h, ph.pair_histogram(A, e))


def test_rejects_bad_edges():
    from paper_2211_00621_gb300 import _lib
    A = synth.sphere_points(5, 10)
    with pytest.raises(_lib.AccelError) as e:
        _gpu(A, np.array([0.5, 0.9], dtype=np.float32))       # not decreasing
    assert e.value.status == 2
    with pytest.raises(_lib.AccelError) as e:
        _gpu(A, np.linspace(0.99, -0.99, 32).astype(np.float32))   # 33 bins
    assert e.value.status == 7
