"""Pins for oracle.pairhist: closed forms (identical points, antipodes, a regular polygon on a
great circle), the union identity of self and cross histograms, and a pure-Python double loop
(CPU only)."""
import math

import numpy as np

from oracle import pairhist as ph
from paper_2211_00621_gb300 import synth


def test_identical_points_fall_in_the_first_bin():
    N = 50
    A = np.tile(np.array([[1.0, 0.0, 0.0]], dtype=np.float32), (N, 1))      # d = 1 exactly
    e = synth.angle_edges(20, 1.0, 10000.0)
    h = ph.pair_histogram(A, e)
    assert h[0] == N * (N - 1) // 2 and h[1:].sum() == 0


def test_antipodal_groups():
    k, m = 9, 6
    A = np.array([[0, 0, 1]] * k + [[0, 0, -1]] * m, dtype=np.float32)
    e = synth.angle_edges(20, 1.0, 10000.0)                 # last edge cos(166.7 deg) > -1
    h = ph.pair_histogram(A, e)
    assert h[0] == k * (k - 1) // 2 + m * (m - 1) // 2
    assert h[-1] == k * m and h[1:-1].sum() == 0


def test_regular_polygon_separations():
    # N points on the equator: separation 2 pi m / N occurs N times (N/2 times for m = N/2);
    # edges at the midpoints cos(pi (2k+1) / N) put separation m into bin m
    for N in (12, 40):
        phi = 2 * np.pi * np.arange(N) / N
        A = np.stack([np.cos(phi), np.sin(phi), np.zeros(N)], axis=1).astype(np.float32)
        e = np.cos(np.pi * (2 * np.arange(N // 2) + 1) / N).astype(np.float32)
        h = ph.pair_histogram(A, e)
        expect = np.zeros(N // 2 + 1, dtype=np.int64)
        expect[1:N // 2] = N
        expect[N // 2] = N // 2
        assert np.array_equal(h, expect)


def test_union_is_self_plus_self_plus_cross():
    A = synth.sphere_points(1, 300)
    B = synth.sphere_points(2, 170)
    e = synth.angle_edges(20, 1.0, 10000.0)
    whole = ph.pair_histogram(np.concatenate([A, B]), e)
    parts = ph.pair_histogram(A, e) + ph.pair_histogram(B, e) + ph.pair_histogram(A, e, B)
    assert np.array_equal(whole, parts)
    assert ph.pair_histogram(A, e, B).sum() == 300 * 170


def test_matches_a_python_double_loop():
    A = synth.sphere_points(3, 60)
    e = synth.angle_edges(12, 30.0, 9000.0)
    h = np.zeros(len(e) + 1, dtype=np.int64)
    f = np.float32
    for i in range(len(A)):
        for j in range(i + 1, len(A)):
            d = f(f(f(A[i, 0]) * f(A[j, 0])) + f(f(A[i, 1]) * f(A[j, 1]))) + f(f(A[i, 2]) * f(A[j, 2]))
            h[sum(1 for x in e if x >= d)] += 1
    assert np.array_equal(ph.pair_histogram(A, e), h)
    assert h.sum() == math.comb(60, 2)
