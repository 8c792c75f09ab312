"""Pins for the oracle's whole step (Sections 2-3).

  * a lone agent follows its preferred velocity (towards the goal at the preferred speed,
    capped by the maximum speed; within one step of the goal it lands on it);
  * far-apart agents do not influence each other;
  * the step commutes with a 180-degree rotation of the scene (exactly: every operation
    maps to its negation) and with a relabelling of agents (no exact distance ties);
  * ORCA's guarantee (Section 3): two agents that see each other, are apart, share tau and
    both find a feasible velocity do not come closer than R within tau;
  * the grid neighbour search gives the same step as brute force.
"""
import numpy as np
import pytest

from paper_1908_10107_gb300 import scenarios as S


def one(**kw):
    base = dict(neighbor_dist=10.0, max_neighbors=10, dt=0.1, knn_mode=0)
    base.update(kw)
    return base


def test_lone_agent_prefers_goal_direction(oracle_mod):
    r = oracle_mod.step(pos=[1, 2], vel=[0, 0], goal=[4, 6], radius=[0.5], max_speed=[2.0],
                        pref_speed=[1.5], time_horizon=[5.0], **one())
    np.testing.assert_allclose(r["vel"][0], [0.9, 1.2], atol=1e-15)
    np.testing.assert_allclose(r["pos"][0], [1.09, 2.12], atol=1e-15)
    # preferred speed above the maximum: capped at the maximum
    r = oracle_mod.step(pos=[1, 2], vel=[0, 0], goal=[4, 6], radius=[0.5], max_speed=[1.0],
                        pref_speed=[1.5], time_horizon=[5.0], **one())
    np.testing.assert_allclose(r["vel"][0], [0.6, 0.8], atol=1e-15)


def test_lone_agent_lands_on_goal(oracle_mod):
    r = oracle_mod.step(pos=[1, 2], vel=[0.3, 0], goal=[1.03, 2.04], radius=[0.5],
                        max_speed=[2.0], pref_speed=[1.0], time_horizon=[5.0], **one())
    np.testing.assert_allclose(r["vel"][0], [0.3, 0.4], atol=1e-14)
    np.testing.assert_allclose(r["pos"][0], [1.03, 2.04], atol=1e-14)


def test_far_agents_do_not_interact(oracle_mod):
    r = oracle_mod.step(pos=[0, 0, 50, 0], vel=[1, 0, -1, 0], goal=[100, 0, -100, 0],
                        radius=[0.5, 0.5], max_speed=[2, 2], pref_speed=[1, 1],
                        time_horizon=[5, 5], **one())
    np.testing.assert_allclose(r["vel"], [[1, 0], [-1, 0]], atol=0)
    assert (r["nbr"] == -1).all()


def _scene(seed, n=300, side=25.0):
    rng = np.random.default_rng(seed)
    return dict(pos=rng.uniform(0, side, (n, 2)).astype(np.float32),
                vel=rng.uniform(-1.5, 1.5, (n, 2)).astype(np.float32),
                goal=rng.uniform(0, side, (n, 2)).astype(np.float32),
                radius=rng.uniform(0.3, 0.5, n).astype(np.float32),
                max_speed=rng.uniform(1.2, 1.6, n).astype(np.float32),
                pref_speed=rng.uniform(1.0, 1.4, n).astype(np.float32),
                time_horizon=np.full(n, 3.0, np.float32))


@pytest.mark.parametrize("seed", range(3))
def test_rotation_by_pi_negates_exactly(oracle_mod, seed):
    sc = _scene(seed)
    kw = dict(neighbor_dist=6.0, max_neighbors=10, dt=0.1, knn_mode=0)
    a = oracle_mod.step(**sc, **kw)
    rot = dict(sc)
    for key in ("pos", "vel", "goal"):
        rot[key] = -sc[key]
    b = oracle_mod.step(**rot, **kw)
    np.testing.assert_array_equal(b["vel"], -a["vel"])
    np.testing.assert_array_equal(b["pos"], -a["pos"])
    np.testing.assert_array_equal(b["nbr"], a["nbr"])
    assert a["lp3"].any() and (~a["lp3"]).any()


@pytest.mark.parametrize("seed", range(3))
def test_relabelling_commutes(oracle_mod, seed):
    sc = _scene(10 + seed)
    kw = dict(neighbor_dist=6.0, max_neighbors=10, dt=0.1, knn_mode=0)
    a = oracle_mod.step(**sc, **kw)
    perm = np.random.default_rng(seed).permutation(len(sc["pos"]))
    inv = np.argsort(perm)
    b = oracle_mod.step(**{k: v[perm] for k, v in sc.items()}, **kw)
    np.testing.assert_array_equal(b["vel"], a["vel"][perm])
    # neighbour j of agent perm[q] appears in b as inv[j]; order is by distance then index,
    # so compare as sets of original labels
    for q in range(0, len(perm), 7):
        got = {int(perm[j]) for j in b["nbr"][q] if j >= 0}
        want = {int(j) for j in a["nbr"][perm[q]] if j >= 0}
        assert got == want


@pytest.mark.parametrize("seed", range(4))
def test_feasible_mutual_pairs_do_not_collide_within_tau(oracle_mod, seed):
    sc = _scene(20 + seed, n=400, side=30.0)
    tau = 3.0
    r = oracle_mod.step(**sc, neighbor_dist=6.0, max_neighbors=12, dt=0.1, knn_mode=0)
    pos = sc["pos"].astype(np.float64)
    rad = sc["radius"].astype(np.float64)
    nbrs = [set(int(j) for j in row if j >= 0) for row in r["nbr"]]
    checked = 0
    for i in range(len(pos)):
        if r["lp3"][i]:
            continue
        for j in nbrs[i]:
            if j <= i or r["lp3"][j] or i not in nbrs[j]:
                continue
            p = pos[j] - pos[i]
            R = rad[i] + rad[j]
            if p @ p <= R * R:
                continue
            dv = r["vel"][j] - r["vel"][i]
            # closest approach of p + dv t over t in [0, tau]
            t = 0.0 if dv @ dv == 0 else np.clip(-(p @ dv) / (dv @ dv), 0.0, tau)
            assert np.linalg.norm(p + dv * t) >= R - 1e-9
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("name", ["circle_swap", "bidirectional", "dense"])
def test_grid_mode_equals_brute_mode(oracle_mod, name):
    sc = S.scene_by_name(name, n=2048 if name != "circle_swap" else 1024)
    sc = S.jitter_velocities(sc, 4)
    a = oracle_mod.step_scene(sc, knn_mode=0)
    b = oracle_mod.step_scene(sc, knn_mode=1)
    np.testing.assert_array_equal(a["nbr"], b["nbr"])
    np.testing.assert_array_equal(a["vel"], b["vel"])
    np.testing.assert_array_equal(a["pos"], b["pos"])


def test_fp64_neighbour_mode_on_exact_floats(oracle_mod):
    """On FP32 positions whose distances are exact in both precisions (a lattice), the FP64
    neighbour search agrees with the FP32 one."""
    g = np.stack(np.meshgrid(np.arange(12.0), np.arange(12.0)), -1).reshape(-1, 2)
    n = len(g)
    sc = dict(pos=g, vel=np.zeros((n, 2)), goal=g + 5, radius=np.full(n, 0.3),
              max_speed=np.full(n, 1.0), pref_speed=np.full(n, 1.0),
              time_horizon=np.full(n, 2.0))
    kw = dict(neighbor_dist=3.5, max_neighbors=8, dt=0.1, knn_mode=1)
    a = oracle_mod.step(**sc, **kw)
    b = oracle_mod.step(**sc, fp64_knn=True, **kw)
    np.testing.assert_array_equal(a["nbr"], b["nbr"])
    np.testing.assert_array_equal(a["vel"], b["vel"])


def test_step_counts_least_penetration_problem_lines(oracle_mod):
    """Two agents overlapping deep inside each other's radius: each one's only half-plane
    lies beyond its speed disc, so LP2 fails at line 0 and the least-penetration LP solves
    one projected problem of one line -- 2 lines over the step.  A lone agent needs no
    fallback (0)."""
    pos = np.array([[0.0, 0.0], [0.3, 0.0]])
    kw = dict(radius=np.full(2, 0.5), max_speed=np.full(2, 1.0), pref_speed=np.full(2, 1.0),
              time_horizon=np.full(2, 2.0), neighbor_dist=5.0, max_neighbors=10, dt=0.1,
              knn_mode=0)
    r = oracle_mod.step(pos, np.zeros((2, 2)), goal=pos + [[10.0, 0.0], [-10.0, 0.0]], **kw)
    assert r["lp3"].all()
    assert r["counters"]["lp3_problem_lines"] == 2
    far = np.array([[0.0, 0.0], [50.0, 0.0]])
    r = oracle_mod.step(far, np.zeros((2, 2)), goal=far + [[10.0, 0.0], [-10.0, 0.0]], **kw)
    assert not r["lp3"].any() and r["counters"]["lp3_problem_lines"] == 0
