"""Pins of the oracle's conditioning tags, which decide which agents the GPU parity gate may
excuse (FP32 against FP64; tests/parity.py).

Two tags exist:
  * margin -- the half-plane construction's discontinuous decisions (agents overlap or not;
    left or right leg of the velocity obstacle, Fig. 1) record their distance to the
    threshold, relative to the quantity's scale; the agent keeps the smallest;
  * sens -- the LP's answer is re-solved with one half-plane at a time shifted along its
    normal by +-4 FP32 ulps of max(|offset|, V) or turned by +-2^-22 rad (the rounding any
    FP32 construction of a half-plane carries); the largest move of the chosen velocity.

Each pin below computes the expected value from geometry written out here (projections,
line intersections, disc chords), not from the oracle's LP, so a wrong ulp scale, a wrong
rotation angle, the wrong line perturbed or a wrong margin scale fails a pin.  An LP whose
optimum sits where two nearly parallel lines cross, or where a line nearly touches the
speed disc, must be tagged; a well-separated vertex must not.
"""
import math

import numpy as np
import pytest

import oracle
from parity import MARGIN, SENS_MAX

ALPHA = 2.0 ** -22  # the rotation of a half-plane in the sensitivity probe (rad)


def eta(c, V):
    """Four FP32 ulps of max(|c|, V): 2^(e-22) for a magnitude in [2^(e-1), 2^e)."""
    return math.ldexp(1.0, math.frexp(max(abs(c), V))[1] - 22)


def line(nx, ny, c):
    """Half-plane n.x >= c (unit n) in the oracle's form [Px, Py, dx, dy]: the boundary
    through P = c n, direction d = (n_y, -n_x), valid side on the left of d."""
    h = math.hypot(nx, ny)
    nx, ny = nx / h, ny / h
    return [c * nx, c * ny, ny, -nx]


def rot(nx, ny, a):
    return nx * math.cos(a) - ny * math.sin(a), nx * math.sin(a) + ny * math.cos(a)


def project_on(nx, ny, c, o):
    """The point of the line n.x = c nearest o (unit n)."""
    s = c - (nx * o[0] + ny * o[1])
    return np.array([o[0] + s * nx, o[1] + s * ny])


def max_move(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def test_single_line_shift_moves_the_answer_by_four_ulps():
    # o violates x >= 1.5 and projects inside the disc's chord: the answer is o's
    # projection, which a shift of the offset moves by exactly the shift
    V, c, o = 1.9, 1.5, (1.0, 0.3)
    s, x = oracle.lp_sensitivity([line(1.0, 0.0, c)], V, o)
    np.testing.assert_allclose(x, [1.5, 0.3], rtol=0, atol=1e-15)
    rot_move = max(max_move(project_on(*rot(1.0, 0.0, a), c, o), x) for a in (ALPHA, -ALPHA))
    want = max(eta(c, V), rot_move)
    assert want == eta(c, V) == 2.0 ** -21
    assert abs(s - want) <= 1e-9 * want
    assert s < SENS_MAX


def test_single_line_turn_dominates_far_from_the_line():
    # o far beyond the line: turning the line by alpha moves the foot of the projection
    # by about (c - n.o) alpha along it, 301.5 * 2^-22 = 7.2e-5 > the tag threshold
    V, c, o = 1.9, 1.5, (-300.0, 0.3)
    s, x = oracle.lp_sensitivity([line(1.0, 0.0, c)], V, o)
    np.testing.assert_allclose(x, [1.5, 0.3], rtol=0, atol=1e-12)
    moves = [max_move(project_on(*rot(1.0, 0.0, a), c, o), x) for a in (ALPHA, -ALPHA)]
    want = max([eta(c, V)] + moves)
    assert abs(want - 301.5 * ALPHA) <= 1e-3 * want
    assert abs(s - want) <= 1e-6 * want
    assert s > SENS_MAX  # tagged


def _vertex(n1, c1, n2, c2):
    A = np.array([n1, n2], float)
    return np.linalg.solve(A, [c1, c2])


@pytest.mark.parametrize("theta", [1e-3, 3e-3])
def test_near_parallel_vertex_is_tagged(theta):
    # two lines crossing at angle theta, o beyond both: the answer is their crossing,
    # which moves by about eta / sin(theta) when either line shifts
    V = 2.0
    n1 = (0.0, 1.0)
    n2 = (-math.sin(theta), math.cos(theta))
    c1, c2 = 0.5, 0.5
    o = (0.0, -1.0)
    lines = [line(*n1, c1), line(*n2, c2)]
    s, x = oracle.lp_sensitivity(lines, V, o)
    np.testing.assert_allclose(x, _vertex(n1, c1, n2, c2), rtol=0, atol=1e-12)
    e = eta(0.5, V)
    moves = []
    for k, (nk, ck) in enumerate(((n1, c1), (n2, c2))):
        for dc in (e, -e):
            m = [(n1, c1), (n2, c2)]
            m[k] = (nk, ck + dc)
            moves.append(max_move(_vertex(m[0][0], m[0][1], m[1][0], m[1][1]), x))
        for a in (ALPHA, -ALPHA):
            m = [(n1, c1), (n2, c2)]
            m[k] = (rot(*nk, a), ck)
            moves.append(max_move(_vertex(m[0][0], m[0][1], m[1][0], m[1][1]), x))
    want = max(moves)
    assert abs(want - e / math.sin(theta)) <= 0.05 * want
    assert abs(s - want) <= 1e-3 * want
    assert s > SENS_MAX  # tagged


def test_near_tangent_line_is_tagged():
    # a line that cuts the speed disc in a chord of half-length h = sqrt(V^2 - c^2) only
    # 7e-3 long; o lies far along it, so the answer is the chord's end, which moves by
    # about c eta / h when the offset shifts
    V = 1.5
    c = V * (1.0 - 1e-5)
    o = (c - 0.2, 50.0)
    s, x = oracle.lp_sensitivity([line(1.0, 0.0, c)], V, o)
    h = math.sqrt(V * V - c * c)
    np.testing.assert_allclose(x, [c, h], rtol=0, atol=1e-9)
    e = eta(c, V)
    moves = [max_move([c + dc, math.sqrt(V * V - (c + dc) ** 2)], x) for dc in (e, -e)]
    want = max(moves)
    assert abs(want - c * e / h) <= 0.05 * want
    assert abs(s - want) <= 1e-6 * want  # the turned lines move the end less
    assert s > SENS_MAX  # tagged


def test_well_separated_vertex_is_not_tagged():
    # perpendicular lines x >= 0.5, y >= 0.3 and o at the origin: the answer is their
    # corner; a shift moves it by exactly the shift, a turn by about |x| alpha
    V = 2.0
    lines = [line(1.0, 0.0, 0.5), line(0.0, 1.0, 0.3)]
    s, x = oracle.lp_sensitivity(lines, V, (0.0, 0.0))
    np.testing.assert_allclose(x, [0.5, 0.3], rtol=0, atol=1e-15)
    want = eta(0.5, V)
    assert want == 2.0 ** -20
    assert abs(s - want) <= 1e-9 * want
    assert s < 0.05 * SENS_MAX


def _equaliser(lines_nc):
    """Least penetration of three half-planes whose normals positively span the plane: the
    unique x where all three penetrations c_i - n_i.x are equal (3x3 linear system)."""
    A = np.array([[nx, ny, 1.0] for (nx, ny), _ in lines_nc])
    b = np.array([c for _, c in lines_nc])
    return np.linalg.solve(A, b)[:2]


def test_least_penetration_answer_is_probed_too():
    # three lines with normals 120 degrees apart and offsets 0.5 have no common point; the
    # least-penetration answer is their equaliser, the origin.  The probe re-runs the LP3
    # fallback on each perturbed problem, so shifting one line moves the answer by 2/3 of
    # the shift along that line's normal
    V = 2.0
    nc = [((math.cos(a), math.sin(a)), 0.5) for a in (0.0, 2 * math.pi / 3, 4 * math.pi / 3)]
    lines = [line(nx, ny, c) for (nx, ny), c in nc]
    used3, x = oracle.solve(lines, V, (0.0, 0.0))
    assert used3
    s, x2 = oracle.lp_sensitivity(lines, V, (0.0, 0.0))
    np.testing.assert_array_equal(x, x2)
    np.testing.assert_allclose(x, [0.0, 0.0], rtol=0, atol=1e-12)
    e = eta(0.5, V)
    moves = []
    for k in range(3):
        for dc in (e, -e):
            m = list(nc)
            m[k] = (nc[k][0], nc[k][1] + dc)
            moves.append(max_move(_equaliser(m), x))
        for a in (ALPHA, -ALPHA):
            m = list(nc)
            m[k] = (rot(*nc[k][0], a), nc[k][1])
            moves.append(max_move(_equaliser(m), x))
    want = max(moves)
    assert abs(want - 2.0 * e / 3.0) <= 1e-6 * want
    assert abs(s - want) <= 1e-6 * want + 1e-13
    assert s < SENS_MAX


def _pair(d, vrel, R, tau, ra_share=0.4):
    """Agents a at the origin and b at (d, 0) with relative velocity v_a - v_b = vrel and
    radius sum R (split ra_share : 1 - ra_share)."""
    ra, rb = R * ra_share, R * (1.0 - ra_share)
    a = [0.0, 0.0, vrel[0], vrel[1], ra]
    b = [d, 0.0, 0.0, 0.0, rb]
    return oracle.orca_line(a, b, tau, 0.1)


@pytest.mark.parametrize("delta", [3e-5, -3e-5, 2e-6, 3e-4])
def test_overlap_decision_margin(delta):
    # |p|^2 = R^2 (1 + delta): the overlap decision is delta (relative) from its threshold;
    # the relative velocity is across p, so the leg decision is far from its own
    R, tau = 1.2, 5.0
    d = R * math.sqrt(1.0 + delta)
    _, _, br, m = _pair(d, (0.0, 1.0), R, tau)
    want = abs(d * d - R * R) / (R * R)
    assert br == (3 if delta < 0 else 1)
    assert abs(m - want) <= 1e-6 * want
    assert (m < MARGIN) == (abs(delta) < MARGIN)


@pytest.mark.parametrize("phi", [2e-5, -7e-5, 0.3])
def test_leg_side_margin(phi):
    # w = v - p/tau at angle phi from p (p = (5, 0), R = 1.2: far apart, w.p > 0 so no
    # cut-off): the left/right leg decision det(p, w) > 0 is |sin phi| from its threshold
    R, tau, d = 1.2, 5.0, 5.0
    wl = 0.5
    w = (wl * math.cos(phi), wl * math.sin(phi))
    vrel = (w[0] + d / tau, w[1])
    _, _, br, m = _pair(d, vrel, R, tau)
    assert br == (1 if phi > 0 else 2)
    overlap_m = (d * d - R * R) / (R * R)
    want = min(abs(math.sin(phi)), overlap_m)
    assert abs(m - want) <= 1e-6 * want
