"""Static obstacles on the GPU against the oracle (the ORCA obstacle rule)."""
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


@pytest.mark.parametrize("steps_before", [0, 40, 150])
def test_bottleneck_matches_the_oracle(steps_before):
    sc = S.bottleneck(1500, seed=31)
    if steps_before == 0:
        sc = S.jitter_velocities(sc, 31)
    rep = parity.gpu_step_and_compare(sc, steps_before=steps_before)
    assert rep["rows"] == sc.n


@pytest.mark.parametrize("tpb", [64, 128])
def test_random_segments_match_the_oracle(tpb):
    rng = np.random.default_rng(32 + tpb)
    sc = S.jitter_velocities(S.bidirectional(3000, seed=33), 33)
    lo, hi = sc.pos.min(0), sc.pos.max(0)
    a = rng.uniform(lo, hi, (60, 2))
    sc.obstacles = np.concatenate([a, a + rng.normal(0, 4, (60, 2))], 1).astype(np.float32)
    sc.obstacle_time_horizon = 3.0
    sim = parity.make_sim(sc)
    abi.orca_set_launch(sim.ctx, tpb, 1)
    rep = parity.gpu_step_and_compare(sc, sim=sim)
    sim.close()
    assert rep["rows"] == sc.n


@pytest.mark.parametrize("steps_before", [0, 120])
def test_bottleneck_far_from_the_origin(steps_before):
    # hundreds of metres out, FP32 coordinates carry ulps of 3e-5 m; the obstacle half-planes
    # of agents pressed into a wall (offset divided by dt) must not inherit them
    sc = S.bottleneck(1500, seed=36)
    shift = np.array([700.0, -450.0], np.float32)
    sc.pos = sc.pos + shift
    sc.goal = sc.goal + shift
    sc.obstacles = sc.obstacles + np.tile(shift, 2)
    if steps_before == 0:
        sc = S.jitter_velocities(sc, 36)
    rep = parity.gpu_step_and_compare(sc, steps_before=steps_before)
    assert rep["rows"] == sc.n


def test_graph_direct_and_launch_shapes_agree_bitwise():
    # the obstacle launch runs beside the plain one (a forked stream inside the step graph);
    # a direct launch, and every launch shape, give the same trajectory
    sc = S.bottleneck(3000, seed=39)
    out = []
    for flags, tpb, lanes in ((0, 0, 0), (abi.ORCA_FLAG_NO_GRAPH, 0, 0), (0, 128, 1),
                              (0, 256, 4), (0, 64, 32)):
        sim = parity.make_sim(sc, flags=flags)
        if tpb:
            abi.orca_set_launch(sim.ctx, tpb, lanes)
        sim.set_scene(sc)
        sim.step(60)
        out.append(sim.get_state())
        sim.close()
    for got in out[1:]:
        np.testing.assert_array_equal(got[0], out[0][0])
        np.testing.assert_array_equal(got[1], out[0][1])


def test_lone_agent_into_a_wall():
    for ang, want in ((np.pi / 2, (0.0, 0.25)), (np.pi / 4, (1.5 / np.sqrt(2.0), 0.25))):
        pos = np.array([[0.0, 0.0]], np.float32)
        goal = np.array([[100.0 * np.cos(ang), 100.0 * np.sin(ang)]], np.float32)
        sc = S.Scene("wall", pos, np.zeros_like(pos), goal, np.full(1, 0.5, np.float32),
                     np.full(1, 3.0, np.float32), np.full(1, 1.5, np.float32),
                     np.full(1, 5.0, np.float32), 10.0, 10, 0.1, 1,
                     obstacles=np.array([[-50.0, 1.0, 50.0, 1.0]], np.float32),
                     obstacle_time_horizon=2.0)
        sim = parity.make_sim(sc)
        sim.set_scene(sc)
        sim.step(1)
        pos2, vel = sim.get_state()
        np.testing.assert_allclose(vel[0], want, atol=1e-5)
        assert sim.get_obstacle_neighbors()[0, 0] == 0
        sim.close()


def test_clearing_obstacles_restores_the_plain_step():
    sc = S.jitter_velocities(S.bidirectional(2000, seed=34), 34)
    plain = parity.make_sim(sc, flags=0)
    plain.set_scene(sc)
    plain.step(3)
    want = plain.get_state()
    plain.close()
    sim = parity.make_sim(sc, flags=0)
    abi.orca_set_obstacles(sim.ctx, np.array([[0.0, 0.0, 1.0, 1.0]], np.float32))
    abi.orca_set_obstacles(sim.ctx, None)
    sim.set_scene(sc)
    sim.step(3)
    got = sim.get_state()
    sim.close()
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


def test_segments_out_of_reach_change_nothing():
    # every tile takes the plain launch; the obstacle launch gets an empty list
    sc = S.jitter_velocities(S.bidirectional(3000, seed=37), 37)
    plain = parity.make_sim(sc)
    plain.set_scene(sc)
    base = abi.orca_launches_per_step(plain.ctx)
    plain.step(4)
    want = plain.get_state()
    plain.close()
    far = sc.copy()
    far.obstacles = np.array([[5000.0, 5000.0, 5010.0, 5000.0], [-900.0, 40.0, -900.0, 80.0]],
                             np.float32)
    sim = parity.make_sim(sc)
    sim.set_scene(far)
    assert abi.orca_launches_per_step(sim.ctx) == base + 2
    sim.step(4)
    got = sim.get_state()
    assert np.all(sim.get_obstacle_neighbors() == -1)
    sim.close()
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])


def test_obstacles_everywhere():
    # a lattice of short walls over the whole crowd: every tile takes the obstacle launch
    sc = S.jitter_velocities(S.bidirectional(2500, seed=38), 38)
    lo, hi = sc.pos.min(0), sc.pos.max(0)
    gx, gy = np.meshgrid(np.linspace(lo[0], hi[0], 16), np.linspace(lo[1], hi[1], 16))
    a = np.stack([gx.ravel(), gy.ravel()], 1)
    sc.obstacles = np.concatenate([a, a + [1.5, 0.5]], 1).astype(np.float32)
    sc.obstacle_time_horizon = np.float32(4.0)
    rep = parity.gpu_step_and_compare(sc, steps_before=5)
    assert rep["rows"] == sc.n


def test_obstacles_are_refused_where_unsupported():
    sc = S.bottleneck(200, seed=35)
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    with pytest.raises(abi.OrcaError):
        abi.orca_count_ops(sim.ctx, True)
    import torch
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(abi.OrcaError):
        abi.orca_rollout_forward(sim.ctx, 4, 2, None, ws)
    with pytest.raises(abi.OrcaError):
        abi.orca_set_obstacles(sim.ctx, np.zeros((300, 4), np.float32))
    sim.close()
