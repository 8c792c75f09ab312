"""Agents leave at their goal (Section 4): the GPU removal against the oracle's arrival rule
on the same FP32 state, and steps after a removal against the oracle."""
import numpy as np
import pytest

import oracle
import parity
from paper_1908_10107_gb300 import abi
from paper_1908_10107_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10107_gb300 import build
    build.build()


def _state_scene(sc, pos, vel):
    st = sc.copy()
    st.pos, st.vel = pos, vel
    return st


def _remove_and_check(sim, sc, kept_so_far):
    """Remove on the GPU; check it against the oracle on the GPU's own state.  Returns the
    compacted scene (oracle view) and the original indices of the survivors."""
    pos, vel = sim.get_state()
    before = _state_scene(sc, pos, vel)
    want_scene, want_keep = oracle.remove_arrived(before)
    m, kept = sim.remove_arrived()
    assert m == want_scene.n
    np.testing.assert_array_equal(kept, want_keep)
    p2, v2 = sim.get_state()
    np.testing.assert_array_equal(p2, pos[want_keep])
    np.testing.assert_array_equal(v2, vel[want_keep])
    return want_scene, kept_so_far[want_keep]


def test_removal_matches_the_oracle_and_steps_continue():
    sc = S.jitter_velocities(S.two_way_crossing(3000, heterogeneous=True, seed=21), 21)
    rng = np.random.default_rng(21)
    # a third of the agents start within their radius of the goal, some exactly on it
    near = rng.choice(sc.n, sc.n // 3, replace=False)
    off = rng.normal(0, 0.5, (near.size, 2)) * sc.radius[near, None]
    sc.goal[near] = (sc.pos[near] + off).astype(np.float32)
    sc.goal[near[:50]] = sc.pos[near[:50]]
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    ids = np.arange(sc.n)
    cur, ids = _remove_and_check(sim, sc, ids)
    assert 0 < cur.n < sc.n
    # the next recorded step (new graph for the new count) matches the oracle
    sim.step(1)
    pos, vel = sim.get_state()
    nbr = sim.get_neighbors()
    cells, gf, gi = sim.get_cells()
    parity.compare_step(cur, pos, vel, nbr, cells, (gf, gi))
    # a few more steps and removals
    for _ in range(3):
        sim.step(5)
        cur, ids = _remove_and_check(sim, cur, ids)
    sim.close()


def test_remove_nobody_and_everybody():
    sc = S.two_way_crossing(500, seed=22)
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    m, kept = sim.remove_arrived()
    assert m == sc.n
    np.testing.assert_array_equal(kept, np.arange(sc.n))
    sim.step(2)
    sc2 = sc.copy()
    sc2.goal = sc2.pos.copy()
    sim.set_scene(sc2)
    m, kept = sim.remove_arrived()
    assert m == 0 and kept.size == 0
    sim.step(3)
    pos, vel = sim.get_state()
    assert pos.shape == (0, 2)
    sim.close()


def test_crossing_runs_until_everybody_arrives():
    sc = S.two_way_crossing(400, seed=23)
    sim = parity.make_sim(sc, flags=0)
    sim.set_scene(sc)
    ids, cur = np.arange(sc.n), sc
    counts = [sc.n]
    for _ in range(400):                 # at most 400 x 10 steps (400 s of crowd time)
        sim.step(10)
        cur, ids = _remove_and_check(sim, cur, ids)
        counts.append(cur.n)
        if cur.n == 0:
            break
    assert counts[-1] == 0, counts[-10:]
    assert all(a >= b for a, b in zip(counts, counts[1:]))
    sim.close()


def test_removal_needs_a_single_scene():
    batch = S.Batch([S.two_way_crossing(200, seed=24), S.two_way_crossing(300, seed=25)])
    sim = abi.OrcaSim.for_batch(batch)
    sim.set_batch(batch)
    with pytest.raises(abi.OrcaError):
        sim.remove_arrived()
    sim.close()


def test_spawn_matches_the_oracle_and_steps_continue():
    """Spawning during a run (Section 4): the candidates the GPU admits are exactly the
    oracle's on the GPU's own state, the entrants are appended at rest with the next agent
    indices, and the step after the spawn matches the oracle."""
    sc = S.two_way_crossing(2500, seed=26)
    sim = parity.make_sim(sc, max_agents=4000)
    sim.set_scene(sc)
    sim.step(60)
    pos, vel = sim.get_state()
    rng = np.random.default_rng(26)
    m = 900
    lo, hi = sc.pos.min(0), sc.pos.max(0)
    cpos = (lo + rng.random((m, 2)) * (hi - lo)).astype(np.float32)
    cgoal = (lo + rng.random((m, 2)) * (hi - lo)).astype(np.float32)
    crad = np.full(m, 0.5, np.float32)
    cpref = np.full(m, 1.0, np.float32)
    cvmax = np.full(m, 1.33, np.float32)
    ctau = np.full(m, 5.0, np.float32)
    window = 1.0
    want = oracle.spawn(pos, vel, sc.radius, cpos, crad, cvmax, window)
    got = sim.spawn(cpos, cgoal, crad, cvmax, cpref, ctau, window)
    np.testing.assert_array_equal(got, want)
    a = int(want.sum())
    assert 0 < a < m and sim.n == sc.n + a
    p2, v2 = sim.get_state()
    np.testing.assert_array_equal(p2[:sc.n], pos)
    np.testing.assert_array_equal(v2[:sc.n], vel)
    np.testing.assert_array_equal(p2[sc.n:], cpos[want])
    assert not v2[sc.n:].any()
    # the crowd with its entrants (oracle view), one recorded step, against the oracle
    st = sc.copy()
    st.pos = np.concatenate([pos, cpos[want]])
    st.vel = np.concatenate([vel, np.zeros((a, 2), np.float32)])
    st.goal = np.concatenate([sc.goal, cgoal[want]])
    st.radius = np.concatenate([sc.radius, crad[want]])
    st.max_speed = np.concatenate([sc.max_speed, cvmax[want]])
    st.pref_speed = np.concatenate([sc.pref_speed, cpref[want]])
    st.time_horizon = np.concatenate([sc.time_horizon, ctau[want]])
    sim.step(1)
    p3, v3 = sim.get_state()
    cells, gf, gi = sim.get_cells()
    parity.compare_step(st, p3, v3, sim.get_neighbors(), cells, (gf, gi))
    sim.close()


def test_spawn_refusals():
    sc = S.two_way_crossing(500, seed=27)
    sim = parity.make_sim(sc, max_agents=600)
    sim.set_scene(sc)
    c = np.zeros((200, 2), np.float32)
    one = np.ones(200, np.float32)
    with pytest.raises(abi.OrcaError) as e:
        sim.spawn(c, c, one, one, one, one, 1.0)
    assert e.value.status == abi.ORCA_ERR_CAPACITY
    sim.close()
    batch = S.Batch([S.two_way_crossing(200, seed=28), S.two_way_crossing(300, seed=29)])
    sim = abi.OrcaSim.for_batch(batch)
    sim.set_batch(batch)
    with pytest.raises(abi.OrcaError) as e:
        sim.spawn(c[:5], c[:5], one[:5], one[:5], one[:5], one[:5], 1.0)
    assert e.value.status == abi.ORCA_ERR_STATE
    sim.close()
