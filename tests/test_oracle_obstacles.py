"""Static obstacles in the oracle (the ORCA obstacle rule: optimisation velocity 0, full
responsibility), pinned to closed forms, to the no-collision guarantee, to exact
arithmetic for the segment selection, and to an LP solver for the hard-line LP3."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1908_10107_gb300 import scenarios as S


def _nc(line4):
    """(n, c) of a line in point-direction form (valid side left of d)."""
    P, d = np.asarray(line4[:2]), np.asarray(line4[2:])
    n = np.array([-d[1], d[0]])
    return n, float(n @ P)


def test_wall_ahead_closed_form():
    line, ov = oracle.obstacle_line((0.0, 0.0), 0.5, (-5.0, 3.0, 5.0, 3.0), 2.0, 0.1)
    assert not ov
    n, c = _nc(line)
    np.testing.assert_allclose(n, [0.0, -1.0], atol=1e-15)
    assert c == pytest.approx(-(3.0 - 0.5) / 2.0, abs=1e-15)      # v_y <= 1.25


def test_nearest_endpoint_closed_form():
    line, _ = oracle.obstacle_line((0.0, 0.0), 0.3, (2.0, 2.0, 4.0, 2.0), 1.5, 0.1)
    n, c = _nc(line)
    np.testing.assert_allclose(n, -np.array([1.0, 1.0]) / np.sqrt(2.0), atol=1e-15)
    assert c == pytest.approx(-(2.0 * np.sqrt(2.0) - 0.3) / 1.5, abs=1e-14)


def test_overlap_pushes_out_within_one_step():
    line, ov = oracle.obstacle_line((0.0, 0.3), 0.5, (-1.0, 0.0, 1.0, 0.0), 2.0, 0.25)
    assert ov
    n, c = _nc(line)
    np.testing.assert_allclose(n, [0.0, 1.0], atol=1e-15)
    assert c == pytest.approx((0.5 - 0.3) / 0.25, abs=1e-14)      # v_y >= 0.8


def _seg_dist(p, seg):
    a, b = np.asarray(seg[:2]), np.asarray(seg[2:])
    e = b - a
    t = np.clip(np.dot(p - a, e) / max(np.dot(e, e), 1e-300), 0.0, 1.0)
    return np.linalg.norm(a + t * e - p)


def test_permitted_velocities_do_not_reach_the_segment_within_tau():
    # the rule's guarantee: a velocity on the permitted side keeps the agent at least r
    # from the segment for the whole time horizon (and the boundary velocity towards the
    # nearest point reaches exactly r at tau)
    rng = np.random.default_rng(5)
    for _ in range(300):
        seg = rng.uniform(-4, 4, 4)
        p = rng.uniform(-4, 4, 2)
        r = rng.uniform(0.2, 0.8)
        tau = rng.uniform(0.5, 4.0)
        if _seg_dist(p, seg) <= r + 1e-3:
            continue
        line, _ = oracle.obstacle_line(p, r, seg, tau, 0.1)
        n, c = _nc(line)
        for _ in range(20):
            v = rng.normal(0, 3, 2)
            if n @ v < c:
                v = v + (c - n @ v + rng.uniform(0, 0.5)) * n      # move onto the permitted side
            ts = np.linspace(0.0, tau, 201)
            d = min(_seg_dist(p + v * t, seg) for t in ts)
            assert d >= r - 1e-9
        q = -n
        vb = c * n                                                  # boundary velocity
        assert _seg_dist(p + vb * tau, seg) == pytest.approx(r, abs=1e-9)


def _selection(pos, seg, radius, vmax, tau_o, k):
    """Nearest reachable segments from exact rational distances on the FP32 inputs (None
    where the FP32 evaluation could round the decision either way)."""
    out = []
    for i in range(pos.shape[0]):
        px, py = (Fraction(float(v)) for v in pos[i])
        rng_ = float(np.float32(np.float32(vmax[i]) * np.float32(tau_o)) + np.float32(radius[i]))
        rng2 = Fraction(float(np.float32(rng_) * np.float32(rng_)))
        ds = []
        for j in range(seg.shape[0]):
            ax, ay, bx, by = (Fraction(float(v)) for v in seg[j])
            ex, ey = bx - ax, by - ay
            l2 = ex * ex + ey * ey
            t = ((px - ax) * ex + (py - ay) * ey) / l2 if l2 else Fraction(0)
            t = min(max(t, Fraction(0)), Fraction(1))
            qx, qy = ax + t * ex - px, ay + t * ey - py
            ds.append((qx * qx + qy * qy, j))
        close = [(d, j) for d, j in ds if d < rng2]
        close.sort()
        sel = [j for _, j in close[:k]]
        # ambiguous if any distance is within rounding of the range or of a neighbour
        vals = sorted(d for d, _ in ds)
        tol = Fraction(1, 10 ** 4) * (rng2 + 1)
        amb = any(abs(d - rng2) < tol for d, _ in ds) or any(
            abs(a - b) < tol for a, b in zip(vals, vals[1:]) if a < rng2)
        out.append(None if amb else sel)
    return out


def test_segment_selection_matches_exact_arithmetic():
    rng = np.random.default_rng(6)
    n, m, k = 300, 40, 4
    pos = rng.uniform(0, 30, (n, 2)).astype(np.float32)
    a = rng.uniform(0, 30, (m, 2))
    seg = np.concatenate([a, a + rng.normal(0, 3, (m, 2))], 1).astype(np.float32)
    sc = S.Scene("obst", pos, np.zeros_like(pos), pos + 1.0, np.full(n, 0.3, np.float32),
                 np.full(n, 1.5, np.float32), np.full(n, 1.0, np.float32), np.full(n, 3.0, np.float32),
                 5.0, 6, 0.1, 1, obstacles=seg, obstacle_time_horizon=2.0, max_obstacle_neighbors=k)
    r = oracle.step_scene(sc, knn_mode=0)
    want = _selection(pos, seg, sc.radius, sc.max_speed, 2.0, k)
    checked = 0
    for i, w in enumerate(want):
        if w is None:
            continue
        got = [j for j in r["obst"][i] if j >= 0]
        assert got == w, i
        checked += 1
    assert checked > 0.8 * n


def test_lp3_keeps_obstacle_lines_hard_and_minimises_the_rest():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(7)
    V, M = 2.0, 512
    ang = np.arange(M) * 2 * np.pi / M
    done = 0
    for _ in range(200):
        nob, nag = rng.integers(1, 3), rng.integers(3, 7)
        lines = []
        for q in range(nob + nag):
            th = rng.uniform(0, 2 * np.pi)
            nrm = np.array([np.cos(th), np.sin(th)])
            c = rng.uniform(-0.6, 0.2) if q < nob else rng.uniform(0.3, 1.8)
            d = np.array([nrm[1], -nrm[0]])
            lines.append([*(c * nrm), *d])
        lines = np.array(lines)
        o = rng.normal(0, 1, 2)
        x, used3 = oracle.solve_fixed(lines, nob, V, o)
        if not used3:
            continue
        nrms = np.stack([-lines[:, 3], lines[:, 2]], 1)
        cs = (nrms * lines[:, :2]).sum(1)
        # hard lines hold
        assert (nrms[:nob] @ x - cs[:nob] >= -1e-9).all()
        assert np.hypot(*x) <= V * (1 + 1e-9)
        # minimax penetration of the other lines subject to the hard ones, on a disc polygon
        A, b = [], []
        for q in range(nob, nob + nag):
            A.append([-nrms[q, 0], -nrms[q, 1], -1.0]); b.append(-cs[q])
        for q in range(nob):
            A.append([-nrms[q, 0], -nrms[q, 1], 0.0]); b.append(-cs[q])
        for t in ang:
            A.append([np.cos(t), np.sin(t), 0.0]); b.append(V)
        res = scipy_opt.linprog([0, 0, 1], A_ub=A, b_ub=b, bounds=[(None, None)] * 3, method="highs")
        if not res.success:
            continue
        pen = max(0.0, (cs[nob:] - nrms[nob:] @ x).max())
        assert pen <= res.x[2] + 2e-3 * V
        done += 1
    assert done > 30


def test_lone_agent_into_a_wall_closed_form():
    # preferred velocity straight at a wall 1 m ahead (r 0.5, tau_o 2): the agent may close
    # at (1 - 0.5)/2 = 0.25 m/s; at 45 degrees it keeps its tangential component
    for ang, want in ((np.pi / 2, (0.0, 0.25)), (np.pi / 4, (1.5 / np.sqrt(2.0), 0.25))):
        pos = np.array([[0.0, 0.0]], np.float32)
        goal = np.array([[100.0 * np.cos(ang), 100.0 * np.sin(ang)]], np.float32)
        sc = S.Scene("wall", pos, np.zeros_like(pos), goal, np.full(1, 0.5, np.float32),
                     np.full(1, 3.0, np.float32), np.full(1, 1.5, np.float32),
                     np.full(1, 5.0, np.float32), 10.0, 10, 0.1, 1,
                     obstacles=np.array([[-50.0, 1.0, 50.0, 1.0]], np.float32),
                     obstacle_time_horizon=2.0)
        r = oracle.step_scene(sc, knn_mode=0)
        np.testing.assert_allclose(r["vel"][0], want, atol=1e-6)
        assert r["obst"][0, 0] == 0
