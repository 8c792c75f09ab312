"""Pins of the oracle's spawning rule (Section 4, test set-up: a new person is placed where it
overlaps nobody within a time window set by size and speed).

Reading: a candidate at rest conflicts with a present agent j when the two could touch within
the window T moving straight at each other, |p_c - p_j| <= r_c + r_j + (V_c + |v_j|) T, and
with an earlier accepted candidate c' likewise with V_c' in place of |v_j|; decided in FP32.
The pins: exact boundary cases built from FP32-exact numbers; the worst case of straight-line
motion sampled over directions; the invariants of the accepted set; order independence of the
crowd; the plain-overlap special case at T = 0.
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_touching_exactly_at_the_reach_is_a_conflict():
    # r_c = 0.25, r_j = 0.75, V_c = 1, |v_j| = |(0.75, 1)| = 1.25, T = 0.5: reach = 1 +
    # 2.25 * 0.5 = 2.125, every quantity exact in FP32
    x = np.float32(2.125)
    up = np.nextafter(x, np.float32(3))
    got = oracle.spawn([[0.0, 0.0]], [[0.75, 1.0]], [0.75], [[x, 0.0], [0.0, -x], [up, 0.0]],
                       [0.25, 0.25, 0.25], [1.0, 1.0, 1.0], 0.5)
    # the first two sit exactly at the reach (conflict); the third one ulp beyond it enters
    # (the first two were rejected, so no earlier accepted candidate blocks it)
    assert got.tolist() == [False, False, True]


def test_earlier_accepted_candidates_block_later_ones():
    # two candidates 3 m apart with r = 0.5 and V = 2 each at T = 0.5: reach 1 + 2 = 3 -> the
    # second conflicts with the first; at 3 m + 1 ulp it enters
    x = np.float32(3.0)
    got = oracle.spawn(np.zeros((0, 2)), np.zeros((0, 2)), [], [[0.0, 0.0], [x, 0.0]],
                       [0.5, 0.5], [2.0, 2.0], 0.5)
    assert got.tolist() == [True, False]
    got = oracle.spawn(np.zeros((0, 2)), np.zeros((0, 2)), [], [[0.0, 0.0], [np.nextafter(x, np.float32(4)), 0.0]],
                       [0.5, 0.5], [2.0, 2.0], 0.5)
    assert got.tolist() == [True, True]
    # a rejected candidate blocks nobody
    got = oracle.spawn([[-2.0, 0.0]], [[0.0, 0.0]], [0.5], [[0.0, 0.0], [x, 0.0]],
                       [0.5, 0.5], [2.0, 2.0], 0.5)
    assert got.tolist() == [False, True]


def test_zero_window_is_plain_overlap():
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 20, (300, 2)).astype(np.float32)
    rad = rng.uniform(0.3, 0.5, 300).astype(np.float32)
    cand = rng.uniform(0, 20, (200, 2)).astype(np.float32)
    crad = rng.uniform(0.3, 0.5, 200).astype(np.float32)
    got = oracle.spawn(pos, rng.normal(size=(300, 2)), rad, cand, crad, np.full(200, 1.5), 0.0)
    d = np.sqrt(((cand[:, None, :].astype(np.float64) - pos[None].astype(np.float64)) ** 2).sum(2))
    overl = (d <= crad[:, None] + rad[None] + 1e-5).any(1)
    clear = (d > crad[:, None] + rad[None] + 1e-5).all(1)
    # away from the rounding margin, a candidate that overlaps a present agent is rejected
    # and one clear of all of them can only be rejected by an earlier accepted candidate
    assert not got[overl].any()
    acc = np.flatnonzero(got)
    for c in np.flatnonzero(clear & ~got):
        dc = np.sqrt(((cand[acc[acc < c]] - cand[c]) ** 2).sum(1))
        assert (dc <= crad[acc[acc < c]] + crad[c] + 1e-5).any()


def _random_case(seed, n=400, m=300, T=0.7):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 40, (n, 2)).astype(np.float32)
    vel = rng.normal(0, 0.8, (n, 2)).astype(np.float32)
    rad = rng.uniform(0.3, 0.5, n).astype(np.float32)
    cand = rng.uniform(0, 40, (m, 2)).astype(np.float32)
    crad = rng.uniform(0.3, 0.6, m).astype(np.float32)
    cv = rng.uniform(1.0, 2.0, m).astype(np.float32)
    return pos, vel, rad, cand, crad, cv, T


def test_accepted_set_is_clear_and_every_rejection_has_a_reason():
    pos, vel, rad, cand, crad, cv, T = _random_case(6)
    got = oracle.spawn(pos, vel, rad, cand, crad, cv, T)
    assert 0 < got.sum() < got.size
    P, C = pos.astype(np.float64), cand.astype(np.float64)
    s = np.sqrt((vel.astype(np.float64) ** 2).sum(1))
    reach_crowd = crad[:, None] + rad[None] + (cv[:, None] + s[None]) * T
    d_crowd = np.sqrt(((C[:, None] - P[None]) ** 2).sum(2))
    acc = np.flatnonzero(got)
    for c in range(len(C)):
        earlier = acc[acc < c]
        reach_c = crad[c] + crad[earlier] + (cv[c] + cv[earlier]) * T
        d_c = np.sqrt(((C[earlier] - C[c]) ** 2).sum(1))
        if got[c]:
            # clear of the crowd and of the earlier accepted ones (FP32 margin)
            assert (d_crowd[c] > reach_crowd[c] * (1 - 1e-6)).all()
            assert (d_c > reach_c * (1 - 1e-6)).all()
        else:
            assert ((d_crowd[c] <= reach_crowd[c] * (1 + 1e-6)).any() or
                    (d_c <= reach_c * (1 + 1e-6)).any())


def test_crowd_order_does_not_matter():
    pos, vel, rad, cand, crad, cv, T = _random_case(7)
    a = oracle.spawn(pos, vel, rad, cand, crad, cv, T)
    p = np.random.default_rng(8).permutation(len(rad))
    b = oracle.spawn(pos[p], vel[p], rad[p], cand, crad, cv, T)
    np.testing.assert_array_equal(a, b)


def test_accepted_candidates_cannot_touch_anyone_within_the_window():
    """The rule's physics: a candidate that enters at rest and then moves at up to V_c in any
    direction stays clear of every present agent moving straight on at its velocity, and
    of every other accepted candidate, for the whole window (directions sampled)."""
    pos, vel, rad, cand, crad, cv, T = _random_case(9, n=200, m=200, T=0.5)
    got = oracle.spawn(pos, vel, rad, cand, crad, cv, T)
    acc = np.flatnonzero(got)
    ang = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    ts = np.linspace(0, T, 21)
    for c in acc:
        for d in dirs:
            pc = cand[c] + ts[:, None] * cv[c] * d[None]  # [t, 2]
            pj = pos[None] + ts[:, None, None] * vel[None]  # [t, n, 2]
            gap = np.sqrt(((pc[:, None] - pj) ** 2).sum(2)) - (crad[c] + rad[None])
            assert gap.min() > -1e-5
