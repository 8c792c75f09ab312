"""Pins for the oracle's spatial bins and neighbour sets (Fig. 2: bins, r_obs filter).

The neighbour rule: the max_neighbors smallest (d^2, j), j != i, d^2 < r_obs^2, with
d^2 taken in FP32 (one rounding per operation).  Pins: an independent numpy brute force
(lexsort over all pairs), the oracle's own grid mode against its brute-force mode,
hand-built tie cases, and geometric containment of cells.
"""
import numpy as np
import pytest

from paper_1908_10107_gb300 import scenarios as S


def numpy_knn(pos, nd, k):
    """Brute force from the definition: all pairs, float32 arithmetic, lexsort by (d2, j)."""
    p = np.asarray(pos, np.float32)
    n = p.shape[0]
    dx = (p[None, :, 0] - p[:, None, 0]).astype(np.float32)
    dy = (p[None, :, 1] - p[:, None, 1]).astype(np.float32)
    d2 = (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
    nd2 = np.float32(nd) * np.float32(nd)
    out = -np.ones((n, k), np.int32)
    for i in range(n):
        j = np.arange(n)
        ok = (j != i) & (d2[i] < nd2)
        jj = j[ok]
        dd = d2[i][ok]
        order = np.lexsort((jj, dd))[:k]
        out[i, : order.size] = jj[order]
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_knn_brute_matches_numpy_definition(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 20, (300, 2)).astype(np.float32)
    for k in (1, 5, 10, 20):
        nbr, _, _ = oracle_mod.knn(pos, 4.0, k, mode=0)
        np.testing.assert_array_equal(nbr, numpy_knn(pos, 4.0, k))


@pytest.mark.parametrize("cell", [0.37, 1.0, 2.5, 4.0, 9.0])
def test_knn_grid_equals_brute(oracle_mod, cell):
    sc = S.bidirectional(4096, seed=5)
    for k in (10, 20):
        gf, gi = oracle_mod.grid(sc.pos, cell, 1 << 22)
        a, da, _ = oracle_mod.knn(sc.pos, sc.neighbor_dist, k, mode=0)
        b, db, _ = oracle_mod.knn(sc.pos, sc.neighbor_dist, k, mode=1, gf=gf, gi=gi)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(da, db)


def test_knn_ties_break_by_index(oracle_mod):
    # A unit lattice: neighbours of the centre at d^2 = 1 (4 of them), 2 (4), 4 (4), 5 (8).
    g = np.stack(np.meshgrid(np.arange(7.0), np.arange(7.0)), -1).reshape(-1, 2)
    rng = np.random.default_rng(3)
    perm = rng.permutation(len(g))
    pos = g[perm].astype(np.float32)
    centre = int(np.where((pos == 3.0).all(1))[0][0])
    nbr, d2, _ = oracle_mod.knn(pos, 10.0, 12, mode=0)
    row, drow = nbr[centre], d2[centre]
    np.testing.assert_array_equal(drow, [1] * 4 + [2] * 4 + [4] * 4)
    for lo in (0, 4, 8):
        assert list(row[lo:lo + 4]) == sorted(row[lo:lo + 4])
    # equal-distance members are exactly the lattice points at that distance
    want1 = {int(np.where((pos == q).all(1))[0][0]) for q in ([2, 3], [4, 3], [3, 2], [3, 4])}
    assert set(row[:4]) == want1


def test_knn_strict_radius_and_padding(oracle_mod):
    pos = np.array([[0, 0], [1, 0], [0, 2], [3, 0]], np.float32)
    nbr, d2, _ = oracle_mod.knn(pos, 2.0, 5, mode=0)
    # d = 2 exactly is excluded (strict <); padding is -1
    assert list(nbr[0]) == [1, -1, -1, -1, -1]
    assert list(nbr[3]) == [-1] * 5
    assert list(nbr[1]) == [0, -1, -1, -1, -1]


def test_knn_circle_swap_neighbours_are_adjacent(oracle_mod):
    sc = S.circle_swap()
    nbr, _, _ = oracle_mod.knn(sc.pos, sc.neighbor_dist, sc.max_neighbors, mode=0)
    n = sc.n
    for i in (0, 1, 511, 1023):
        got = set(int(j) for j in nbr[i])
        want = {(i + d) % n for d in (-5, -4, -3, -2, -1, 1, 2, 3, 4, 5)}
        assert got == want


def test_cells_contain_agents(oracle_mod):
    sc = S.dense(20000, seed=9)
    for cell, cap in ((1.0, 1 << 30), (0.25, 5000)):
        gf, gi = oracle_mod.grid(sc.pos, cell, cap)
        gx, gy = int(gi[0]), int(gi[1])
        assert gx * gy <= cap
        s = float(gf[2])
        # capacity rule: the edge is the smallest power-of-two multiple that fits
        assert s >= cell
        if s > cell:
            ext = sc.pos.max(0).astype(np.float64) - sc.pos.min(0)
            assert (np.floor(ext[0] / (s / 2)) + 1) * (np.floor(ext[1] / (s / 2)) + 1) > cap
        c = oracle_mod.cells(sc.pos, gf, gi)
        cx, cy = c % gx, c // gx
        assert c.max() < gx * gy
        x = sc.pos[:, 0].astype(np.float64) - gf[0]
        y = sc.pos[:, 1].astype(np.float64) - gf[1]
        tol = 1e-5 * (s + np.abs(sc.pos).max())
        assert np.all(x >= cx * s - tol) and np.all(x <= (cx + 1) * s + tol)
        assert np.all(y >= cy * s - tol) and np.all(y <= (cy + 1) * s + tol)
