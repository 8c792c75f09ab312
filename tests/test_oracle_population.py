"""Arrival and removal (Section 4: a person who reaches the goal location leaves the
simulation) in the oracle, pinned to exact arithmetic and to the step's own behaviour."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1908_10107_gb300 import scenarios as S


def _one(p, g, r):
    return bool(oracle.arrived(np.array([p], np.float32), np.array([g], np.float32),
                               np.array([r], np.float32))[0])


def test_boundary_cases():
    assert _one((2.0, 3.0), (2.0, 3.0), 0.5)             # at the goal
    assert _one((0.0, 0.0), (0.5, 0.0), 0.5)             # exactly one radius away
    assert not _one((0.0, 0.0), (np.nextafter(np.float32(0.5), np.float32(1)), 0.0), 0.5)
    assert _one((0.0, 0.0), (3.0, 4.0), 5.0)             # 3-4-5, on the boundary
    assert not _one((0.0, 0.0), (3.0, 4.0), np.nextafter(np.float32(5), np.float32(0)))
    assert not _one((0.0, 0.0), (100.0, 0.0), 0.5)


def test_matches_exact_arithmetic_away_from_the_boundary():
    # exact rational |goal - p|^2 against r^2 on the FP32 inputs, wherever the two differ
    # by more than the rounding of the FP32 evaluation
    rng = np.random.default_rng(3)
    n = 4000
    p = (rng.uniform(-500, 500, (n, 2))).astype(np.float32)
    g = (p + rng.normal(0, 0.6, (n, 2))).astype(np.float32)
    r = rng.uniform(0.3, 1.0, n).astype(np.float32)
    got = oracle.arrived(p, g, r)
    checked = 0
    for i in range(n):
        d2 = (Fraction(float(g[i, 0])) - Fraction(float(p[i, 0]))) ** 2 + \
             (Fraction(float(g[i, 1])) - Fraction(float(p[i, 1]))) ** 2
        r2 = Fraction(float(r[i])) ** 2
        if abs(d2 - r2) > Fraction(1, 10 ** 4) * r2 + Fraction(1, 10 ** 6):
            assert got[i] == (d2 <= r2), i
            checked += 1
    assert checked > 0.9 * n and 0.1 * n < got.sum() < 0.9 * n


def test_removal_keeps_order_and_parameters():
    sc = S.two_way_crossing(400, heterogeneous=True, seed=9)
    sc.goal[::3] = sc.pos[::3]                            # every third agent is at its goal
    out, keep = oracle.remove_arrived(sc)
    assert out.n == sc.n - len(range(0, sc.n, 3))
    assert np.all(np.diff(keep) > 0) and not np.any(keep % 3 == 0)
    for name in ("pos", "vel", "goal", "radius", "max_speed", "pref_speed", "time_horizon"):
        np.testing.assert_array_equal(getattr(out, name), getattr(sc, name)[keep])
    sc.goal[:] = sc.pos
    empty, keep = oracle.remove_arrived(sc)
    assert empty.n == 0 and keep.size == 0


def test_an_agent_within_one_step_of_its_goal_arrives_after_the_step():
    # the preferred velocity steps onto the goal when it is within pref_speed * dt, and a
    # lone agent takes its preferred velocity, so after one step it has arrived
    for d in (0.05, 0.09, 0.1):
        pos = np.array([[10.0, -3.0]], np.float32)
        goal = (pos + np.array([[d * 0.6, d * 0.8]])).astype(np.float32)
        sc = S.Scene("one", pos, np.zeros_like(pos), goal, np.full(1, 0.2, np.float32),
                     np.full(1, 1.5, np.float32), np.full(1, 1.0, np.float32),
                     np.full(1, 5.0, np.float32), 10.0, 10, 0.1, 1)
        r = oracle.step_scene(sc, knn_mode=0)
        assert oracle.arrived(r["pos"].astype(np.float32), goal, sc.radius)[0]
        assert not oracle.arrived(pos, goal, np.full(1, 0.04, np.float32))[0]
