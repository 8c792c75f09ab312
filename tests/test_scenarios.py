"""The seeded workload generators (shared by the GPU path and the oracle)."""
import numpy as np

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
