"""Pins for the oracle's 2-D linear program and its least-penetration fallback (Section 3).

LP2: the point of {|x| <= V} intersected with the half-planes {det(d_i, x - P_i) >= 0}
closest to o (or, in direction mode, the point maximising o.x).  The minimiser of a
strictly convex objective is unique, so any correct method must return it: pinned by
brute-force enumeration of every candidate optimum (o itself, projections of o on each
line and on the circle, line-line and line-circle intersections).

LP3: when the half-planes miss the disc, the velocity minimising the largest violation
max_i det(d_i, P_i - x) over the disc.  The optimal value is pinned by scipy's HiGHS
solver on the same minimax written as an LP, with the disc replaced by circumscribed and
inscribed 4096-gons that bracket it.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linprog

TOL = 1e-9


def feasible(x, lines, V, tol=TOL):
    if np.linalg.norm(x) > V + tol:
        return False
    for P, d in lines:
        if d[0] * (x[1] - P[1]) - d[1] * (x[0] - P[0]) < -tol:
            return False
    return True


def line_circle(P, d, V):
    a = P @ d
    D = a * a + V * V - P @ P
    if D < 0:
        return []
    s = np.sqrt(D)
    return [P + (-a - s) * d, P + (-a + s) * d]


def line_line(P1, d1, P2, d2):
    den = d1[0] * d2[1] - d1[1] * d2[0]
    if abs(den) < 1e-12:
        return []
    # P1 + t d1 = P2 + s d2
    t = ((P2[0] - P1[0]) * d2[1] - (P2[1] - P1[1]) * d2[0]) / den
    return [P1 + t * d1]


def enumerate_lp(lines, V, o, dir_opt):
    o = np.asarray(o, float)
    cands = []
    if not dir_opt:
        cands.append(o.copy())
        for P, d in lines:
            cands.append(P + ((o - P) @ d) * d)
        no = np.linalg.norm(o)
        if no > 0:
            cands.append(o * (V / no))
    else:
        cands.append(o * V)
    for P, d in lines:
        cands += line_circle(P, d, V)
    for (P1, d1), (P2, d2) in itertools.combinations(lines, 2):
        cands += line_line(P1, d1, P2, d2)
    feas = [c for c in cands if feasible(c, lines, V)]
    if not feas:
        return None
    if dir_opt:
        return max(feas, key=lambda c: c @ o)
    return min(feas, key=lambda c: np.linalg.norm(c - o))


def random_lines(rng, n, V):
    lines = []
    for _ in range(n):
        ang = rng.uniform(0, 2 * np.pi)
        d = np.array([np.cos(ang), np.sin(ang)])
        P = rng.uniform(-1.2 * V, 1.2 * V, 2)
        lines.append((P, d))
    return lines


def pack(lines):
    return np.array([[P[0], P[1], d[0], d[1]] for P, d in lines], float).reshape(-1, 4)


@pytest.mark.parametrize("seed", range(4))
def test_lp2_matches_vertex_enumeration(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n_feas = n_infeas = 0
    for trial in range(400):
        n = int(rng.integers(0, 7))
        V = rng.uniform(0.5, 2.5)
        lines = random_lines(rng, n, V)
        o = rng.uniform(-2 * V, 2 * V, 2)
        ret, x = oracle_mod.lp2(pack(lines), V, o, False)
        best = enumerate_lp(lines, V, o, False)
        if best is None:
            assert ret < n
            n_infeas += 1
            continue
        if ret < n:
            # reported infeasible although a point exists: only allowed for a region
            # thinner than the parallel-line tolerance
            assert all(feasible(best, lines, V, 1e-9) for _ in [0])
            continue
        n_feas += 1
        np.testing.assert_allclose(x, best, atol=1e-9)
        assert feasible(x, lines, V, 1e-9)
    assert n_feas > 200 and n_infeas > 20


@pytest.mark.parametrize("seed", range(3))
def test_lp2_direction_mode_matches_enumeration(oracle_mod, seed):
    rng = np.random.default_rng(50 + seed)
    checked = 0
    for _ in range(300):
        n = int(rng.integers(0, 6))
        V = rng.uniform(0.5, 2.5)
        lines = random_lines(rng, n, V)
        ang = rng.uniform(0, 2 * np.pi)
        o = np.array([np.cos(ang), np.sin(ang)])
        ret, x = oracle_mod.lp2(pack(lines), V, o, True)
        best = enumerate_lp(lines, V, o, True)
        if best is None or ret < n:
            assert (best is None) == (ret < n) or best is None
            continue
        checked += 1
        assert feasible(x, lines, V, 1e-9)
        assert abs(x @ o - best @ o) <= 1e-9
    assert checked > 100


def minimax_bounds(lines, V, m=4096):
    """HiGHS on min t s.t. det(d_i, P_i - x) <= t, x in a regular m-gon (two radii)."""
    out = []
    for radius in (V / np.cos(np.pi / m), V):  # circumscribed, inscribed polygon
        A, b = [], []
        for P, d in lines:
            # det(d, P - x) = d0 (P1 - x1) - d1 (P0 - x0) <= t
            A.append([d[1], -d[0], -1.0])
            b.append(-(d[0] * P[1] - d[1] * P[0]))
        th = 2 * np.pi * np.arange(m) / m
        # vertices at angles th; edges: x.n_k <= radius * cos(pi/m), n_k at th + pi/m
        nk = th + np.pi / m
        for c, s in zip(np.cos(nk), np.sin(nk)):
            A.append([c, s, 0.0])
            b.append(radius * np.cos(np.pi / m))
        res = linprog([0, 0, 1], A_ub=np.array(A), b_ub=np.array(b),
                      bounds=[(None, None)] * 3, method="highs")
        assert res.status == 0
        out.append(res.fun)
    return out[0], out[1]


@pytest.mark.parametrize("seed", range(4))
def test_lp3_reaches_minimax_penetration(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    done = 0
    for _ in range(120):
        n = int(rng.integers(2, 11))
        V = rng.uniform(0.5, 2.0)
        lines = []
        for _ in range(n):
            ang = rng.uniform(0, 2 * np.pi)
            d = np.array([np.cos(ang), np.sin(ang)])
            # push lines outwards so the constraint set often misses the disc
            P = rng.uniform(-3 * V, 3 * V, 2)
            lines.append((P, d))
        o = rng.uniform(-V, V, 2)
        lp3_used, x = oracle_mod.solve(pack(lines), V, o)
        if not lp3_used:
            continue
        pen = max(d[0] * (P[1] - x[1]) - d[1] * (P[0] - x[0]) for P, d in lines)
        lo, hi = minimax_bounds(lines, V)
        assert hi > -1e-9  # infeasible set really has positive minimax penetration
        assert np.linalg.norm(x) <= V + 1e-9
        assert lo - 1e-7 <= pen <= hi + 1e-7, (lo, pen, hi)
        done += 1
    assert done > 40


def test_lp3_single_unreachable_line(oracle_mod):
    """One line entirely outside the disc: the least-penetration point is V times the
    line's inward normal (the disc point closest to the half-plane)."""
    V = 1.5
    line = np.array([[0.0, 3.0, 1.0, 0.0]])  # valid side: y >= 3 (left of (1, 0))
    used, x = oracle_mod.solve(line, V, [0.3, -0.2])
    assert used
    np.testing.assert_allclose(x, [0.0, V], atol=1e-15)


def test_lp_feasible_result_satisfies_all_constraints(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(500):
        n = int(rng.integers(1, 12))
        V = rng.uniform(0.5, 2.0)
        lines = random_lines(rng, n, V)
        o = rng.uniform(-2, 2, 2)
        used, x = oracle_mod.solve(pack(lines), V, o)
        if not used:
            # feasible case: every half-plane and the speed bound hold to 1e-9
            assert feasible(x, lines, V, 1e-9)
        else:
            # least-penetration case: nearly parallel lines make the projected LP
            # ill-conditioned; the speed bound holds to rounding of that LP
            assert np.linalg.norm(x) <= V * (1 + 1e-7)


def test_lp3_problem_lines_closed_forms(oracle_mod):
    """The count of lines in LP3's projected problems (a problem for line i, 0-based,
    takes that line and the i before it).  Closed forms: n parallel lines facing the same
    way, each farther outside the disc than the last, open one problem each (every line is
    violated by more than the penetration the previous problem reached, and same-direction
    bisectors constrain nothing), so the count is 1 + 2 + ... + n; a feasible LP opens
    none; two opposite parallel lines with a gap fail LP2 at the second and open one
    problem of two lines, whose optimum is the midline."""
    V = 1.0
    for n in (1, 2, 3, 5, 10):
        # valid side x >= 1.5 + 0.1 i: normal (1, 0), direction (0, -1)
        lines = np.array([[1.5 + 0.1 * i, 0.0, 0.0, -1.0] for i in range(n)])
        used, x, c = oracle_mod.solve_counted(lines, V, [0.0, 0.0])
        assert used
        assert c["lp3_problem_lines"] == n * (n + 1) // 2
        np.testing.assert_allclose(x, [V, 0.0], atol=1e-15)
    feasible_lines = np.array([[-0.5, 0.0, 0.0, -1.0], [0.0, -0.5, 1.0, 0.0]])  # x >= -0.5, y >= -0.5
    used, x, c = oracle_mod.solve_counted(feasible_lines, V, [0.2, 0.1])
    assert not used and c["lp3_problem_lines"] == 0
    np.testing.assert_allclose(x, [0.2, 0.1], atol=1e-15)
    gap = np.array([[0.5, 0.0, 0.0, -1.0], [-0.5, 0.0, 0.0, 1.0]])  # x >= 0.5, x <= -0.5
    used, x, c = oracle_mod.solve_counted(gap, V, [0.0, 0.0])
    assert used and c["lp3_problem_lines"] == 2
    np.testing.assert_allclose(x[0], 0.0, atol=1e-15)
