"""GPU step vs the FP64 oracle through the C ABI (parity tests proper).

Sizes span many 128-agent tiles with ragged tails; the full-size workloads are checked on
sampled agents (the oracle steps only those, searching neighbours among all agents).
"""
import numpy as np
import pytest

from paper_1908_10107_gb300 import abi
from paper_1908_10107_gb300 import scenarios as S

import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10107_gb300 import build
    build.build()


@pytest.mark.parametrize("steps_before", [0, 10, 60])
def test_circle_swap_1024(steps_before):
    rep = parity.gpu_step_and_compare(S.circle_swap(), steps_before=steps_before)
    assert rep["rows"] == 1024


@pytest.mark.parametrize("n,seed", [(16381, 1), (4099, 2)])
@pytest.mark.parametrize("jitter", [False, True])
def test_bidirectional_small(n, seed, jitter):
    sc = S.bidirectional(n, seed=seed)
    if jitter:
        sc = S.jitter_velocities(sc, seed)
    parity.gpu_step_and_compare(sc)


@pytest.mark.parametrize("steps_before", [0, 1500])
def test_eight_way_crossing(steps_before):
    """The paper's eight-way crossing (Section 4, Fig. 5) at its 10,000 agents: at the start
    and after 1,500 steps (150 s), when the eight crowds meet in the vortex near the centre."""
    sc = S.eight_way_crossing(10000)
    rep = parity.gpu_step_and_compare(sc, steps_before=steps_before)
    assert rep["rows"] == 10000


@pytest.mark.parametrize("heterogeneous", [False, True])
def test_two_way_crossing(heterogeneous):
    """The paper's two-way crossing (Section 4, Figs. 3-4) at its 2,500 agents, equal and
    varied agents, when the two crowds meet."""
    sc = S.two_way_crossing(2500, heterogeneous=heterogeneous)
    rep = parity.gpu_step_and_compare(sc, steps_before=400)
    assert rep["rows"] == 2500


def test_bidirectional_after_steps():
    sc = S.bidirectional(8190, seed=3)
    parity.gpu_step_and_compare(sc, steps_before=40)


def test_dispersing_neighbours_outrun_the_predicted_radius():
    # a nearly stationary agent among fast agents running radially outwards (1 m per
    # step): its k-th neighbour distance grows far beyond the radius predicted from the
    # previous step, so the neighbour search must fall back to the r_obs bound
    rng = np.random.default_rng(41)
    m = 40
    ang = rng.uniform(0.0, 2.0 * np.pi, m)
    rad = rng.uniform(1.0, 3.0, m)
    ring = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    pos = np.concatenate([[[0.0, 0.0]], ring]).astype(np.float32)
    goal = np.concatenate([[[0.0, 0.0]], ring / rad[:, None] * 1e4]).astype(np.float32)
    vmax = np.concatenate([[0.01], np.full(m, 60.0)]).astype(np.float32)
    sc = S.Scene("dispersing", pos, np.zeros_like(pos), goal, np.full(m + 1, 0.2, np.float32),
                 vmax, vmax.copy(), np.full(m + 1, 2.0, np.float32), 50.0, 10, 1.0 / 60.0, 1)
    for steps_before in (1, 4):
        rep = parity.gpu_step_and_compare(sc, steps_before=steps_before)
        assert rep["rows"] == m + 1


@pytest.mark.parametrize("k", [10, 20])
def test_dense_small(k):
    sc = S.dense(20011, seed=4)
    sc.max_neighbors = k
    sc = S.jitter_velocities(sc, 5)
    parity.gpu_step_and_compare(sc)


@pytest.mark.parametrize("cell_size", [0.3, 1.0, 2.5, 10.0, 40.0])
def test_cell_size_does_not_change_results(cell_size):
    sc = S.jitter_velocities(S.bidirectional(6000, seed=6), 6)
    parity.gpu_step_and_compare(sc, cell_size=cell_size)


@pytest.mark.parametrize("spacing,steps_before", [(3.0, 0), (3.0, 3), (6.0, 0), (6.0, 3)])
def test_sparse_lattice_with_tiny_cells(spacing, steps_before):
    # cells far smaller than the neighbour distances: with no radius prediction the search
    # starts from the local density (few agents in the 3 x 3 tiny cells) and grows the
    # radius 1.5x many times; at spacing 6 most agents have fewer than k = 10 neighbours
    # inside r_obs = 10 (the prediction then says so)
    rng = np.random.default_rng(int(spacing * 10) + steps_before)
    g = np.stack(np.meshgrid(np.arange(24.0), np.arange(24.0)), -1).reshape(-1, 2) * spacing
    g = g + rng.uniform(-0.2, 0.2, g.shape)
    sc = _tiny(g, r=0.4, nd=10.0, dt=0.1)
    sc = S.jitter_velocities(sc, 7)
    rep = parity.gpu_step_and_compare(sc, cell_size=0.05, steps_before=steps_before)
    assert rep["rows"] == g.shape[0]


def test_cell_capacity_doubling():
    sc = S.jitter_velocities(S.bidirectional(5000, seed=7), 7)
    parity.gpu_step_and_compare(sc, cell_size=0.1, max_cells=1000)


@pytest.mark.parametrize("k", [1, 3, 16, 32])
def test_neighbour_counts(k):
    sc = S.jitter_velocities(S.dense(3000, seed=8), 8)
    sc.max_neighbors = k
    parity.gpu_step_and_compare(sc)


def test_full_size_bidirectional_sampled():
    sc = S.bidirectional()  # 524,288 agents, the benchmark's workload
    rng = np.random.default_rng(0)
    subset = np.sort(rng.choice(sc.n, 4000, replace=False))
    parity.gpu_step_and_compare(sc, steps_before=5, subset=subset)


@pytest.mark.parametrize("cell,tpb,lanes", [(1.4105, 64, 1), (1.7631, 64, 1), (1.4105, 128, 32)])
def test_full_size_bidirectional_in_the_benchmarked_launch_shapes(cell, tpb, lanes):
    """The 524,288-agent flow in the settings the benchmark's tuner picks among (cell edges
    1.41 / 1.76 m, 64 threads with one lane per solve, 128 threads with warp work units),
    after 20 steps (the benchmark's warm-up), sampled."""
    sc = S.bidirectional()
    sim = parity.make_sim(sc, cell_size=cell)
    abi.orca_set_launch(sim.ctx, tpb, lanes)
    subset = np.sort(np.random.default_rng(int(cell * 1000) + tpb).choice(sc.n, 3000, replace=False))
    rep = parity.gpu_step_and_compare(sc, steps_before=20, cell_size=cell, sim=sim, subset=subset)
    sim.close()
    assert rep["rows"] == len(subset)


def test_full_size_dense_sampled():
    sc = S.dense()  # 2,097,152 agents, k = 20
    rng = np.random.default_rng(1)
    subset = np.sort(rng.choice(sc.n, 2000, replace=False))
    parity.gpu_step_and_compare(sc, subset=subset)


# ----------------------------------------------------------------------------- edge cases
def _tiny(pos, vel=None, goal=None, r=0.5, vmax=1.5, pref=1.0, tau=5.0, nd=10.0, k=10, dt=0.1):
    pos = np.asarray(pos, np.float32).reshape(-1, 2)
    n = pos.shape[0]
    f = lambda v: np.full(n, v, np.float32)
    return S.Scene("tiny", pos, np.zeros_like(pos) if vel is None else np.asarray(vel, np.float32).reshape(-1, 2),
                   (pos + 5.0) if goal is None else np.asarray(goal, np.float32).reshape(-1, 2),
                   f(r), f(vmax), f(pref), f(tau), nd, k, dt, 1)


def test_empty_crowd():
    sim = parity.make_sim(_tiny(np.zeros((1, 2))))
    abi.orca_set_agents(sim.ctx, 0, *[np.zeros(0, np.float32)] * 7)
    sim.step(3)
    pos, vel = sim.get_state()
    assert pos.shape == (0, 2)
    sim.sync()


def test_single_agent():
    parity.gpu_step_and_compare(_tiny([[1.0, 2.0]], goal=[[4.0, 6.0]]))


def test_head_on_pair():
    sc = _tiny([[-2.0, 0.0], [2.0, 0.0]], vel=[[1.0, 0.0], [-1.0, 0.0]],
               goal=[[1000.0, 0.0], [-1000.0, 0.0]], vmax=1.33, pref=1.0, tau=10.0, dt=0.25)
    parity.gpu_step_and_compare(sc)


def test_coincident_agents():
    pos = np.array([[0, 0], [0, 0], [0, 0], [0.3, 0.0], [5, 5]], np.float32)
    parity.gpu_step_and_compare(_tiny(pos))


def test_all_agents_in_one_cell():
    sc = S.jitter_velocities(S.bidirectional(1500, seed=9), 9)
    parity.gpu_step_and_compare(sc, cell_size=1e4)


def test_neighbour_radius_is_strict():
    # lattice spacing 2.0 with r_obs 2.0: the axis neighbours at exactly r_obs are excluded
    g = np.stack(np.meshgrid(np.arange(20.0), np.arange(20.0)), -1).reshape(-1, 2) * 2.0
    sc = _tiny(g, nd=2.0, r=0.3)
    parity.gpu_step_and_compare(sc)
    sc = _tiny(g, nd=2.0001, r=0.3)
    parity.gpu_step_and_compare(sc)


def test_lattice_ties_break_by_index():
    g = np.stack(np.meshgrid(np.arange(30.0), np.arange(30.0)), -1).reshape(-1, 2)
    perm = np.random.default_rng(10).permutation(len(g))
    sc = _tiny(g[perm], nd=3.0, r=0.2, k=12)
    parity.gpu_step_and_compare(sc)


# ------------------------------------------------------------------- determinism, readout
def test_graph_and_direct_launch_agree_bitwise():
    sc = S.jitter_velocities(S.bidirectional(10000, seed=11), 11)
    out = []
    for flags in (0, abi.ORCA_FLAG_NO_GRAPH):
        sim = parity.make_sim(sc, flags=flags)
        sim.set_scene(sc)
        sim.step(25)
        out.append(sim.get_state())
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_state_round_trip_is_exact():
    sc = S.jitter_velocities(S.dense(7000, seed=12), 12)
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    pos, vel = sim.get_state()
    np.testing.assert_array_equal(pos, sc.pos)
    np.testing.assert_array_equal(vel, sc.vel)
    sim.step(7)
    pos, vel = sim.get_state()
    # resume from a checkpoint: reload the read-out state, continue, compare with uninterrupted
    st = sc.copy()
    st.pos, st.vel = pos, vel
    sim2 = parity.make_sim(sc)
    sim2.set_scene(st)
    sim.step(5)
    sim2.step(5)
    a, b = sim.get_state(), sim2.get_state()
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_device_pointers_match_host_pointers():
    import torch
    sc = S.jitter_velocities(S.bidirectional(5000, seed=13), 13)
    sim = parity.make_sim(sc)
    dev = [torch.from_numpy(a).cuda() for a in sc.arrays()]
    sim.set_agents(*dev)
    sim.step(3)
    pd, vd = sim.get_state(device=True)
    torch.cuda.synchronize()
    sim.set_scene(sc)
    sim.step(3)
    ph, vh = sim.get_state()
    np.testing.assert_array_equal(pd.cpu().numpy(), ph)
    np.testing.assert_array_equal(vd.cpu().numpy(), vh)


def test_search_counters():
    """The first step after a load starts every search without a prediction; later steps
    start from the previous k-th neighbour distance.  On a sparse lattice with tiny cells
    the start radius must grow: extra passes are counted."""
    sc = S.bidirectional(8190, seed=41)
    sim = parity.make_sim(sc, flags=0)
    sim.set_scene(sc)
    sim.step(1)
    c1 = sim.search_counters()
    assert c1["unpredicted"] == sc.n and c1["rows"] >= 2 * sc.n
    sim.step(3)
    c4 = sim.search_counters()
    assert c4["unpredicted"] == sc.n  # no new unpredicted searches
    assert c4["rows"] > c1["rows"]
    sim.close()
    g = np.stack(np.meshgrid(np.arange(24.0), np.arange(24.0)), -1).reshape(-1, 2) * 6.0
    lat = _tiny(g, r=0.4, nd=10.0, dt=0.1)
    sim = parity.make_sim(lat, flags=0, cell_size=0.05)
    sim.set_scene(lat)
    sim.step(1)
    assert sim.search_counters()["extra_passes"] > 0
    sim.close()


def test_counters():
    sc = S.jitter_velocities(S.bidirectional(4000, seed=14), 14)
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    sim.step(4)
    c = sim.counters()
    assert c["agent_steps"] == 4 * sc.n
    assert 0 < c["lp3_agent_steps"] <= c["agent_steps"]
    assert c["lines"] <= 4 * sc.n * sc.max_neighbors
    assert c["candidates"] >= c["lines"]


@pytest.mark.parametrize("scene", ["flow", "dense20", "circle"])
def test_lp_modes_agree_bitwise(scene):
    # one lane per agent, the agent split and warp work units take the same decisions
    # with the same roundings: identical states after several steps, and the same
    # least-penetration work (the lines of the projected problems each mode solved)
    if scene == "flow":
        sc = S.jitter_velocities(S.bidirectional(8190, seed=17), 17)
    elif scene == "dense20":
        sc = S.dense(20011, seed=18)
        sc.max_neighbors = 20
        sc = S.jitter_velocities(sc, 18)
    else:
        sc = S.circle_swap()
    states, work = {}, {}
    for tpb, lanes in ((64, 1), (64, 4), (128, 4), (64, 32), (256, 32)):
        sim = parity.make_sim(sc, flags=0)
        abi.orca_set_launch(sim.ctx, tpb, lanes)
        sim.set_scene(sc)
        sim.step(12)
        states[(tpb, lanes)] = sim.get_state()
        work[(tpb, lanes)] = sim.search_counters()["lp3_problem_lines"]
        sim.close()
    ref = states[(64, 1)]
    for key, (pos, vel) in states.items():
        np.testing.assert_array_equal(pos, ref[0], err_msg=str(key))
        np.testing.assert_array_equal(vel, ref[1], err_msg=str(key))
        assert work[key] == work[(64, 1)], (key, work)
    assert scene == "circle" or work[(64, 1)] > 0


@pytest.mark.parametrize("scene,tpb", [("two_way", 64), ("eight_way", 128), ("dense20", 64)])
def test_agent_split_passes_parity(scene, tpb):
    """Four lanes per agent (neighbour search, half-planes and least penetration shared by a
    quad of lanes): exact neighbour lists and cells, velocities within the oracle's bar."""
    if scene == "two_way":
        sc = S.two_way_crossing(2500, heterogeneous=True)
    elif scene == "eight_way":
        sc = S.eight_way_crossing(10000)
    else:
        sc = S.dense(6007, seed=19)
        sc.max_neighbors = 20
        sc = S.jitter_velocities(sc, 19)
    sim = parity.make_sim(sc)
    abi.orca_set_launch(sim.ctx, tpb, 4)
    rep = parity.gpu_step_and_compare(sc, steps_before=30, sim=sim)
    sim.close()
    assert rep["rows"] == sc.n


def test_operation_counts_match_the_oracle():
    # the counting launch counts the LP operations the oracle counts on the same state
    # (they can differ only where an FP32 decision differs from the FP64 one), and
    # counting changes no result
    import oracle
    sc = S.jitter_velocities(S.bidirectional(8190, seed=16), 16)
    ref = oracle.step_scene(sc, knn_mode=1)["counters"]
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    abi.orca_count_ops(sim.ctx, True)
    sim.step(1)
    ops, c = sim.op_counters(), sim.counters()
    plines = sim.search_counters()["lp3_problem_lines"]
    pos, vel = sim.get_state()
    sim.close()
    assert c["lines"] == ref["lines"]
    # every step counts the lines of the least-penetration projected problems
    assert ref["lp3_problem_lines"] > 0
    assert abs(plines - ref["lp3_problem_lines"]) <= 0.01 * ref["lp3_problem_lines"], \
        (plines, ref["lp3_problem_lines"])
    assert abs(c["lp3_agent_steps"] - ref["lp3_agents"]) <= 0.002 * sc.n
    for key in ("lp1_calls", "lp1_bounds", "lp_checks", "bisectors"):
        assert ref[key] > 0
        assert abs(ops[key] - ref[key]) <= 0.01 * ref[key], (key, ops[key], ref[key])
    plain = parity.make_sim(sc)
    plain.set_scene(sc)
    plain.step(1)
    assert not any(plain.op_counters().values())
    p2, v2 = plain.get_state()
    plain.close()
    np.testing.assert_array_equal(pos, p2)
    np.testing.assert_array_equal(vel, v2)


def test_non_finite_input_is_reported():
    sc = _tiny(np.random.default_rng(15).uniform(0, 10, (64, 2)))
    sc.pos[3] = np.nan
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    sim.step(1)
    with pytest.raises(abi.OrcaError) as e:
        sim.sync()
    assert e.value.status == abi.ORCA_ERR_NUMERIC


def test_capacity_errors():
    sc = _tiny(np.zeros((10, 2)))
    sim = parity.make_sim(sc, max_agents=5)
    with pytest.raises(abi.OrcaError) as e:
        sim.set_scene(sc)
    assert e.value.status == abi.ORCA_ERR_CAPACITY
    sim2 = parity.make_sim(sc, flags=0)
    sim2.set_scene(sc)
    with pytest.raises(abi.OrcaError) as e:
        sim2.get_neighbors()
    assert e.value.status == abi.ORCA_ERR_STATE
