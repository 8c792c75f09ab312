"""The seeded workload generators (shared by the GPU path and the oracle)."""
import numpy as np
import pytest

from paper_1908_10107_gb300 import scenarios as S


def test_seeded_and_fp32():
    a, b = S.bidirectional(4096, seed=3), S.bidirectional(4096, seed=3)
    for x, y in zip(a.arrays(), b.arrays()):
        assert x.dtype == np.float32
        np.testing.assert_array_equal(x, y)
    assert a.dt == float(np.float32(1 / 60))


def test_bidirectional_shape():
    sc = S.bidirectional(524288)
    x = sc.pos[:, 0]
    h = sc.n // 2
    assert x[:h].min() >= 0 and x[:h].max() <= 250
    assert x[h:].min() >= 750 and x[h:].max() <= 1000
    np.testing.assert_allclose(sc.goal[:h, 0] - sc.pos[:h, 0], 750, atol=1e-3)
    assert 0.3 <= sc.radius.min() and sc.radius.max() <= 0.5
    np.testing.assert_array_equal(sc.max_speed, sc.pref_speed)


def test_circle_swap_shape():
    sc = S.circle_swap()
    np.testing.assert_allclose(np.linalg.norm(sc.pos, axis=1), 100.0, rtol=1e-6)
    np.testing.assert_array_equal(sc.goal, -sc.pos)


def test_batch_counts_log_uniform():
    b = S.batched()
    counts = np.array([s.n for s in b.scenes])
    assert len(counts) == 256 and counts.min() >= 500 and counts.max() <= 50000
    # log-uniform: the median count is near the geometric mean of the range
    assert 2000 < np.median(counts) < 12000
    off = b.offsets
    assert off[-1] == b.n == sum(a.shape[0] for a in b.arrays()[:1])
    kinds = {s.name for s in b.scenes}
    assert kinds == {"circle_swap", "bidirectional"}


def _min_gap(sc):
    """Smallest (distance - r_i - r_j - c_i - c_j) over all pairs (brute force)."""
    p = sc.pos.astype(np.float64)
    span = sc.radius.astype(np.float64) + sc.pref_speed.astype(np.float64) * sc.dt
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    gap = d - span[:, None] - span[None, :]
    np.fill_diagonal(gap, np.inf)
    return gap.min()


@pytest.mark.parametrize("heterogeneous", [False, True])
def test_two_way_crossing_layout(heterogeneous):
    sc = S.two_way_crossing(1200, heterogeneous=heterogeneous, seed=5)
    assert sc.n == 1200 and _min_gap(sc) >= -1e-4  # spawned without overlap (float32 storage)
    h = sc.n // 2
    # crowd A starts left of the origin and heads right, crowd B the other way; each
    # crowd's goals lie in the other's start region
    assert (sc.pos[:h, 0] < 0).all() and (sc.pos[h:, 0] > 0).all()
    for a, b in ((slice(0, h), slice(h, None)), (slice(h, None), slice(0, h))):
        lo, hi = sc.pos[b].min(0), sc.pos[b].max(0)
        assert (sc.goal[a] >= lo - 1.5).all() and (sc.goal[a] <= hi + 1.5).all()
    if heterogeneous:
        assert set(np.unique(sc.radius)) == {np.float32(0.5), np.float32(0.75), np.float32(1.0)}
        assert set(np.unique(sc.pref_speed)) == {np.float32(1.0), np.float32(1.33), np.float32(2.0)}
        np.testing.assert_allclose(sc.max_speed, 1.25 * sc.pref_speed.astype(np.float64), rtol=1e-6)
    else:
        assert (sc.radius == np.float32(0.5)).all() and (sc.pref_speed == np.float32(1.0)).all()
        assert (sc.max_speed == np.float32(1.33)).all()
    again = S.two_way_crossing(1200, heterogeneous=heterogeneous, seed=5)
    np.testing.assert_array_equal(sc.pos, again.pos)
    np.testing.assert_array_equal(sc.goal, again.goal)


def test_eight_way_crossing_layout():
    sc = S.eight_way_crossing(2000, seed=6)
    assert sc.n == 2000 and _min_gap(sc) >= -1e-4
    ang = np.arctan2(sc.pos[:, 1].astype(np.float64), sc.pos[:, 0])
    gang = np.arctan2(sc.goal[:, 1].astype(np.float64), sc.goal[:, 0])
    m = sc.n // 8
    for c in range(8):
        rows = slice(c * m, (c + 1) * m)
        start = np.angle(np.exp(1j * ang[rows]).mean())
        turn = np.angle(np.exp(1j * gang[rows]).mean() / np.exp(1j * start))
        # the crowd starts at 45-degree step c and heads 135 degrees further round
        assert abs(np.angle(np.exp(1j * (start - c * np.pi / 4)))) < 0.05
        assert abs(turn - 3 * np.pi / 4) < 0.05


def test_spawn_rejects_a_full_region():
    rng = np.random.default_rng(0)
    lo, hi = np.zeros((50, 2)), np.full((50, 2), 3.0)
    with pytest.raises(ValueError):
        S.spawn_without_overlap(rng, lo, hi, np.full(50, 0.5), np.zeros(50), max_tries=50)


def test_bottleneck_layout():
    sc = S.bottleneck(800, seed=7)
    assert sc.obstacles.dtype == np.float32 and sc.obstacles.shape == (4, 4)
    assert sc.max_obstacle_neighbors == 4 and sc.obstacle_time_horizon == np.float32(2.0)
    # the door: the two wall pieces on x = 0 leave a gap of the door's width around y = 0
    wall = sc.obstacles[:2]
    assert np.all(wall[:, [0, 2]] == 0.0)
    assert np.isclose(wall[1, 1] - wall[0, 3], 2.4)
    # every agent in the room, clear of every wall by its radius, and the spawn discs apart
    h = sc.obstacles[0, 1]
    assert np.all(sc.pos[:, 0] < -sc.radius) and np.all(np.abs(sc.pos[:, 1]) < -h - sc.radius)
    d = np.linalg.norm(sc.pos[:, None].astype(np.float64) - sc.pos[None], axis=2)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2 * sc.radius.max()
    # goals past the door, within its width across
    assert np.all(sc.goal[:, 0] >= 10.0) and np.all(np.abs(sc.goal[:, 1]) <= 0.4 * 2.4 + 1e-6)


def test_two_way_stream_spawn_source():
    empty, src = S.two_way_stream(400, seed=3)
    assert empty.n == 0 and src.n == 400
    rng = np.random.default_rng(0)
    pos, goal, rad, vmax, pref, tau = src.candidates(rng)
    assert pos.dtype == np.float32 and pos.shape == (400, 2)
    assert np.all(pos >= src.lo - 1e-4) and np.all(pos <= src.hi + 1e-4)
    # the two crowds start on opposite sides and head for each other's region
    assert np.all(np.sign(pos[:200, 0]) == -np.sign(goal[:200, 0]))
    mask = np.zeros(400, bool)
    mask[::3] = True
    src.admit(mask)
    assert src.n == 400 - mask.sum()
    assert src.candidates(rng)[0].shape == (src.n, 2)
