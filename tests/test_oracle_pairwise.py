"""Pins for oracle.pairwise: two-body closed form, symmetric configurations and zero net
momentum (CPU only)."""
import itertools
import math

import numpy as np
import pytest

from oracle import pairwise
from paper_2211_00621_gb300 import synth


def test_two_body_closed_form():
    eps = 1e-3
    pos = np.array([[0.1, 0.2, 0.3], [0.4, -0.2, 0.3]])
    m = np.array([2.0, 3.0])
    a = pairwise.accel(pos, m, eps)
    r = math.sqrt(0.3 ** 2 + 0.4 ** 2)  # = 0.5
    s = (r * r + eps * eps) ** 1.5
    # body 0 is pulled towards body 1 with magnitude m1 r / (r^2 + eps^2)^(3/2)
    np.testing.assert_allclose(a[0], 3.0 * np.array([0.3, -0.4, 0.0]) / s, rtol=1e-14)
    np.testing.assert_allclose(a[1], 2.0 * np.array([-0.3, 0.4, 0.0]) / s, rtol=1e-14)


def test_cube_corners_cancel_at_centre():
    corners = np.array(list(itertools.product([0.0, 1.0], repeat=3)))
    pos = np.vstack([corners, [[0.5, 0.5, 0.5]]])
    m = np.concatenate([np.full(8, 1.3), [0.7]])
    a = pairwise.accel(pos, m, 1e-3)
    assert np.abs(a[8]).max() < 1e-14
    # each corner is pulled towards the inside along the diagonal: all components equal size
    for c in range(8):
        d = np.sign(0.5 - corners[c])
        assert np.all(a[c] * d > 0)
        np.testing.assert_allclose(np.abs(a[c]), np.abs(a[c])[0], rtol=1e-13)


def test_self_term_is_zero_and_eps_softening():
    # a single body feels nothing; two coincident bodies feel nothing.
    assert np.abs(pairwise.accel(np.zeros((1, 3)), np.ones(1), 1e-3)).max() == 0.0
    assert np.abs(pairwise.accel(np.zeros((2, 3)), np.ones(2), 1e-3)).max() == 0.0


def test_zero_net_momentum():
    b = synth.bodies(0, 300)
    a = pairwise.accel(b["pos"], b["mass"], 1e-3)
    net = (b["mass"][:, None] * a).sum(axis=0)
    scale = (b["mass"][:, None] * np.abs(a)).sum()
    assert np.abs(net).max() < 1e-13 * scale


def test_subset_matches_full():
    b = synth.bodies(1, 100)
    full = pairwise.accel(b["pos"], b["mass"], 1e-3)
    idx = [0, 17, 99]
    np.testing.assert_array_equal(pairwise.accel(b["pos"], b["mass"], 1e-3, idx), full[idx])
    assert pairwise.term_scale(b["pos"], b["mass"], 1e-3, idx).shape == (3,)


def test_term_scale_two_bodies_hand_worked():
    # (0,0,0) m=2 and (3,0,0) m=5, eps=4: r^2 + eps^2 = 9 + 16 = 25, 25^(3/2) = 125; the self
    # term is zero; each body sees the other's |m_j r / (r^2+eps^2)^(3/2)| = m_j 3 / 125, then
    # divided by sqrt(N) = sqrt(2)
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    got = pairwise.term_scale(pos, np.array([2.0, 5.0]), 4.0, [0, 1])
    np.testing.assert_allclose(got, [0.0848528137423857029, 0.0339411254969542812], rtol=1e-14)


def test_term_scale_three_bodies_hand_worked():
    # a 3-4-5 right triangle, masses 1, 2, 3, eps = 4: the denominators are 25^1.5 = 125,
    # 32^1.5 = 181.01933598375617 and 41^1.5 = 262.52809373474680; body 0 sums 2*3/125 +
    # 3*4/181.019..., body 1 1*3/125 + 3*5/262.528..., body 2 1*4/181.019... + 2*5/262.528...,
    # each divided by sqrt(3)
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    got = pairwise.term_scale(pos, np.array([1.0, 2.0, 3.0]), 4.0, [0, 1, 2])
    np.testing.assert_allclose(got, [0.0659860901520891945, 0.0468443199239936631, 0.0347497013859574824],
                               rtol=1e-14)


def test_term_scale_bounds_the_acceleration():
    # |a_i| <= sum_j |term_ij| (triangle inequality), with equality when every other body lies
    # on one ray from i (all terms parallel): collinear bodies on one side
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [2.5, 0.0, 0.0], [4.0, 0.0, 0.0]])
    m = np.array([1.0, 2.0, 0.5, 3.0])
    n = len(m)
    a0 = np.linalg.norm(pairwise.accel(pos, m, 0.1, [0])[0])
    np.testing.assert_allclose(pairwise.term_scale(pos, m, 0.1, [0])[0] * np.sqrt(n), a0, rtol=1e-14)
    b = synth.bodies(4, 50)
    a = np.linalg.norm(pairwise.accel(b["pos"], b["mass"], 1e-3), axis=1)
    ts = pairwise.term_scale(b["pos"], b["mass"], 1e-3, range(50)) * np.sqrt(50)
    assert np.all(a <= ts * (1 + 1e-12))
