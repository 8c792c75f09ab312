"""Pins for the oracle's ORCA half-plane (Fig. 1 a-c).

The half-plane of agent a induced by b is built from u, the shortest vector from the
relative velocity v = v_a - v_b to the boundary of the truncated velocity obstacle
VO^tau = union over t in (0, tau] of the discs D(p/t, R/t), p = p_b - p_a, R = r_a + r_b.
Its boundary passes through v_a + u/2 and its valid side faces along the outward normal
of VO at v + u.

Pins, none of which reuse the oracle's leg/cutoff formulas:
  * the VO distance by direct minimisation over the family of discs (exterior points)
    and by the support function of the convex set VO (interior points);
  * hand-derived closed forms for a head-on pair, a resting pair inside the cut-off
    range, and a resting overlapping pair.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def vo_nearest_boundary(p, v, R, tau):
    """(inside, distance, outward unit normal at the nearest boundary point)."""
    p = np.asarray(p, float)
    v = np.asarray(v, float)
    pn = np.linalg.norm(p)

    def f(s):  # signed distance from v to disc D(s p, s R), s = 1/t >= 1/tau
        return np.linalg.norm(v - s * p) - s * R

    s_lo = 1.0 / tau
    s_hi = s_lo + 10.0 * (np.linalg.norm(v) + 10.0 * R + pn) / (pn - R)
    grid = np.linspace(s_lo, s_hi, 20001)
    vals = np.linalg.norm(v[None, :] - grid[:, None] * p[None, :], axis=1) - grid * R
    i = int(np.argmin(vals))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    res = minimize_scalar(f, bounds=(a, b), method="bounded", options={"xatol": 1e-15})
    s_best, f_best = (res.x, res.fun) if res.fun < vals[i] else (grid[i], vals[i])
    if f_best >= 0.0:
        c = s_best * p
        nrm = (v - c) / np.linalg.norm(v - c)
        return False, f_best, nrm
    # interior: distance = min over admissible outward normals e of h(e) - v.e,
    # h(e) = (p.e + R)/tau for p.e + R <= 0 (support function of the convex VO)
    alpha = math.acos(R / pn)
    base = math.atan2(-p[1], -p[0])

    def g(phi):
        e = np.array([math.cos(base + phi), math.sin(base + phi)])
        return (p @ e + R) / tau - v @ e

    phis = np.linspace(-alpha, alpha, 200001)
    es = np.stack([np.cos(base + phis), np.sin(base + phis)], 1)
    gv = ((es @ p) + R) / tau - es @ v
    i = int(np.argmin(gv))
    a, b = phis[max(i - 1, 0)], phis[min(i + 1, len(phis) - 1)]
    res = minimize_scalar(g, bounds=(a, b), method="bounded", options={"xatol": 1e-15})
    phi = res.x if res.fun < gv[i] else phis[i]
    return True, min(res.fun, gv[i]), np.array([math.cos(base + phi), math.sin(base + phi)])


def left_normal(line):
    return np.array([-line[3], line[2]])


@pytest.mark.parametrize("seed", range(6))
def test_u_is_shortest_vector_to_vo_boundary(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    checked = {0: 0, 1: 0, 2: 0}
    for _ in range(60):
        R = rng.uniform(0.6, 1.2)
        tau = rng.uniform(1.0, 10.0)
        ang = rng.uniform(0, 2 * np.pi)
        dist = rng.uniform(1.05 * R, 8.0 * R)
        p = dist * np.array([np.cos(ang), np.sin(ang)])
        vrel = rng.uniform(-3, 3, 2)
        a = [0.0, 0.0, vrel[0], vrel[1], R / 2]
        b = [p[0], p[1], 0.0, 0.0, R / 2]
        line, u, br, margin = oracle_mod.orca_line(a, b, tau, 0.1)
        assert br in (0, 1, 2)
        inside, d, nrm = vo_nearest_boundary(p, vrel, R, tau)
        if d < 1e-6:
            continue
        assert abs(np.linalg.norm(u) - d) <= 1e-7 * max(1.0, d), (br, inside)
        # u points to the nearest boundary point: outward when inside, inward when outside
        expect_u = d * nrm if inside else -d * nrm
        np.testing.assert_allclose(u, expect_u, atol=2e-5 * max(1.0, d))
        # valid side faces the outward normal; the boundary passes through v_a + u/2
        np.testing.assert_allclose(left_normal(line), nrm, atol=2e-5)
        np.testing.assert_allclose(line[:2], np.array(a[2:4]) + u / 2, atol=1e-12)
        assert abs(np.linalg.norm(line[2:]) - 1.0) < 1e-12
        checked[br] += 1
    assert sum(checked.values()) > 40


@pytest.mark.parametrize("seed", range(3))
def test_overlap_uses_one_step_disc(oracle_mod, seed):
    """Overlapping agents: u reaches the boundary of D(p/dt, R/dt) (sampled circle)."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        R = rng.uniform(0.6, 1.2)
        dt = rng.choice([0.25, 0.1, 1 / 60])
        ang = rng.uniform(0, 2 * np.pi)
        p = rng.uniform(0.05, 0.95) * R * np.array([np.cos(ang), np.sin(ang)])
        vrel = rng.uniform(-3, 3, 2)
        line, u, br, _ = oracle_mod.orca_line([0, 0, vrel[0], vrel[1], R / 2],
                                              [p[0], p[1], 0, 0, R / 2], 5.0, dt)
        assert br == 3
        th = np.linspace(0, 2 * np.pi, 400001)
        circle = p / dt + (R / dt) * np.stack([np.cos(th), np.sin(th)], 1)
        dists = np.linalg.norm(circle - vrel, axis=1)
        i = int(np.argmin(dists))
        assert abs(np.linalg.norm(u) - dists[i]) < 1e-6 * (R / dt)
        np.testing.assert_allclose(vrel + u, circle[i], atol=1e-4 * (R / dt))
        inside = np.linalg.norm(vrel - p / dt) < R / dt
        out_n = (circle[i] - p / dt) / (R / dt)
        np.testing.assert_allclose(left_normal(line), out_n, atol=1e-4)
        assert inside == (u @ out_n > 0)


def _load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_head_on_pair_closed_form(oracle_mod):
    """Two agents with the paper's two-way-crossing parameters meet head on.

    A at (-d, 0) moving +x at s, B at (d, 0) moving -x at s, R = 2r.  Derivation: v = (2s, 0),
    p = (2d, 0); w = v - p/tau has w.p > 0 when s*tau > d, so the leg case applies; det(p, w)
    = 0 selects the right leg, whose direction is (-l, R)/(2d), l = sqrt(4d^2 - R^2); u is
    the component of -v normal to it, u = (-sR^2, -s l R)/(2d^2).  The preferred velocity
    equals v_a, whose projection on the line is v_a + u/2, so
        v_a' = (s - sR^2/(4d^2), -s l R/(4d^2)),   v_b' = -v_a'.
    """
    g = _load_golden("paper_agent_parameters.json")["two_way_crossing_uniform"]
    r, s, vmax = g["radius_m"], g["desired_speed_mps"], g["max_speed_mps"]
    d, tau, dt = 2.0, 10.0, 0.25
    R = 2 * r
    l = math.sqrt(4 * d * d - R * R)
    want = np.array([s - s * R * R / (4 * d * d), -s * l * R / (4 * d * d)])
    res = oracle_mod.step(pos=[-d, 0, d, 0], vel=[s, 0, -s, 0], goal=[1000, 0, -1000, 0],
                          radius=[r, r], max_speed=[vmax, vmax], pref_speed=[s, s],
                          time_horizon=[tau, tau], neighbor_dist=15.0, max_neighbors=10,
                          dt=dt, knn_mode=0)
    np.testing.assert_allclose(res["vel"][0], want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(res["vel"][1], -want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(res["pos"][0], [-d, 0] + want * dt, atol=1e-14)
    assert not res["lp3"].any()


def test_resting_pair_cutoff_closed_form(oracle_mod):
    """A at rest, B at rest at distance d > R: cut-off case.  w = -p/tau, n = -p/|p|,
    u = ((d - R)/tau, 0); the constraint is x <= (d - R)/(2 tau).  With a preferred
    velocity (s, 0) above that bound, v_a' = ((d - R)/(2 tau), 0)."""
    d, R, tau, s = 3.0, 1.0, 2.0, 1.0
    res = oracle_mod.step(pos=[0, 0, d, 0], vel=[0, 0, 0, 0], goal=[100, 0, d, 0],
                          radius=[R / 2, R / 2], max_speed=[2.0, 2.0], pref_speed=[s, s],
                          time_horizon=[tau, tau], neighbor_dist=10.0, max_neighbors=4,
                          dt=0.1, knn_mode=0)
    np.testing.assert_allclose(res["vel"][0], [(d - R) / (2 * tau), 0.0], atol=1e-15)


@pytest.mark.parametrize("dt,vmax", [(0.25, 2.0), (1 / 60, 1.5)])
def test_resting_overlap_closed_form(oracle_mod, dt, vmax):
    """Resting agents overlapping by R - e: each must leave D(p/dt, R/dt), i.e. move apart at
    (R - e)/(2 dt).  When that exceeds the maximum speed the constraint cannot be met and
    the least-penetration velocity is full speed straight away from the other agent."""
    R, e = 1.0, 0.5
    res = oracle_mod.step(pos=[0, 0, e, 0], vel=[0, 0, 0, 0], goal=[0, 0, e, 0],
                          radius=[R / 2, R / 2], max_speed=[vmax, vmax], pref_speed=[1, 1],
                          time_horizon=[5, 5], neighbor_dist=10.0, max_neighbors=4, dt=dt,
                          knn_mode=0)
    need = (R - e) / (2 * dt)
    sp = min(need, vmax)
    np.testing.assert_allclose(res["vel"][0], [-sp, 0.0], atol=1e-12)
    np.testing.assert_allclose(res["vel"][1], [sp, 0.0], atol=1e-12)
    assert bool(res["lp3"][0]) == (need > vmax)
