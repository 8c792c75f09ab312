"""Batched scenes through orca_set_scenes: every scene of the batch against the oracle run on
that scene alone, and bitwise against the same scene stepped in a context of its own."""
import numpy as np
import pytest

import oracle
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


def small_batch(seed=0, sizes=(1500, 37, 2900, 1, 640, 0, 2048, 999, 313, 1200, 128, 2500)):
    rng = np.random.default_rng(seed)
    scenes = []
    for s, n in enumerate(sizes):
        if s % 3 == 0:
            sc = S.circle_swap(max(n, 1), circle_radius=100.0 * max(n, 1) / 1024.0)
        elif s % 3 == 1:
            sc = S.bidirectional(max(n, 1), seed=seed + s)
        else:
            sc = S.dense(max(n, 1), seed=seed + s)
            sc.max_neighbors = int(rng.choice([5, 16, 20]))
        if n == 0:
            sc = S.Scene(sc.name, sc.pos[:0], sc.vel[:0], sc.goal[:0], sc.radius[:0], sc.max_speed[:0],
                         sc.pref_speed[:0], sc.time_horizon[:0], sc.neighbor_dist, sc.max_neighbors,
                         sc.dt, 1)
        scenes.append(S.jitter_velocities(sc, seed + s) if n > 0 else sc)
    return S.Batch(scenes)


def run_batch(batch, steps_before=0, flags=abi.ORCA_FLAG_RECORD):
    sim = abi.OrcaSim.for_batch(batch, flags=flags)
    sim.set_batch(batch)
    if steps_before:
        sim.step(steps_before)
    return sim


def check_batch_against_oracle(sim, batch, max_cells, scenes=None, sample=None):
    off = batch.offsets
    sim.step(1)
    pos, vel = sim.get_state()
    nbr = sim.get_neighbors()
    cells, _, _ = sim.get_cells()
    gf, gi = sim.get_scene_grids()
    reports = []
    for s in (range(len(batch.scenes)) if scenes is None else scenes):
        sc = batch.scenes[s]
        a, b = int(off[s]), int(off[s + 1])
        if b == a:
            continue
        k = sc.max_neighbors
        local = nbr[a:b, :k].copy()
        local[local >= 0] -= a
        assert (nbr[a:b, k:] == -1).all()
        budget = max(1, max_cells * sc.n // batch.n)
        rows = None if sample is None else np.sort(np.random.default_rng(s).choice(sc.n, min(sample, sc.n), replace=False))
        rep = parity.compare_step(
            sc, pos[a:b], vel[a:b], local, (cells[a:b] - gi[s, 2]).astype(np.uint32),
            (gf[s], gi[s, :2]), cell_size=0.0, max_cells=budget, subset=rows)
        reports.append(rep)
    return reports


def test_small_batch_against_oracle():
    batch = small_batch()
    sim = run_batch(batch)
    before = batch  # step 0 from the loaded state
    reps = check_batch_against_oracle(sim, before, max_cells=max(4 * batch.n, 65536))
    assert len(reps) == 11


def test_small_batch_after_steps():
    batch = small_batch(seed=5)
    sim = run_batch(batch, steps_before=12)
    pos, vel = sim.get_state()
    off = batch.offsets
    cur = S.Batch([sc.copy() for sc in batch.scenes])
    for s, sc in enumerate(cur.scenes):
        sc.pos, sc.vel = pos[off[s]:off[s + 1]].copy(), vel[off[s]:off[s + 1]].copy()
    check_batch_against_oracle(sim, cur, max_cells=max(4 * batch.n, 65536))


def test_scene_in_batch_equals_scene_alone_bitwise():
    # the same states, and so the same least-penetration work: the batch's count of
    # projected-problem lines is the sum of the scenes' counts stepped alone
    batch = small_batch(seed=9)
    sim = run_batch(batch, flags=0)
    sim.step(20)
    pos, vel = sim.get_state()
    batch_work = sim.search_counters()["lp3_problem_lines"]
    off = batch.offsets
    alone_work = 0
    for s, sc in enumerate(batch.scenes):
        if sc.n == 0:
            continue
        alone = abi.OrcaSim.for_scene(sc)
        alone.set_scene(sc)
        alone.step(20)
        p1, v1 = alone.get_state()
        alone_work += alone.search_counters()["lp3_problem_lines"]
        alone.close()
        np.testing.assert_array_equal(pos[off[s]:off[s + 1]], p1)
        np.testing.assert_array_equal(vel[off[s]:off[s + 1]], v1)
    assert batch_work == alone_work > 0


def test_batch_state_update_rescans_the_boxes_bitwise():
    """After steps, every scene's grid comes from the box the ORCA kernel reduced for it;
    new positions written from outside (orca_update_state) invalidate those boxes, and the
    next step must scan: stepping on equals a fresh batch loaded with the new state, bit
    for bit (grids included)."""
    batch = small_batch(seed=11)
    sim = run_batch(batch, steps_before=6)
    pos, vel = sim.get_state()
    pos = (pos + np.float32(0.37)).astype(np.float32)
    sim.update_state(pos, vel)
    sim.step(3)
    p1, v1 = sim.get_state()
    g1 = sim.get_scene_grids()
    off = batch.offsets
    fresh = S.Batch([sc.copy() for sc in batch.scenes])
    for s, sc in enumerate(fresh.scenes):
        sc.pos, sc.vel = pos[off[s]:off[s + 1]].copy(), vel[off[s]:off[s + 1]].copy()
    ref = run_batch(fresh, steps_before=3)
    p2, v2 = ref.get_state()
    g2 = ref.get_scene_grids()
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(v1, v2)
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a, b)
    sim.close()
    ref.close()


def test_default_batch_sampled():
    batch = S.batched()  # 256 scenes, ~2.6M agents
    sim = run_batch(batch, steps_before=3)
    pos, vel = sim.get_state()
    off = batch.offsets
    cur = S.Batch([sc.copy() for sc in batch.scenes])
    for s, sc in enumerate(cur.scenes):
        sc.pos, sc.vel = pos[off[s]:off[s + 1]].copy(), vel[off[s]:off[s + 1]].copy()
    order = np.argsort([sc.n for sc in batch.scenes])
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1]), 7, 100, 200]
    check_batch_against_oracle(sim, cur, max_cells=max(4 * batch.n, 65536), scenes=pick, sample=600)


def test_batch_argument_checks():
    batch = small_batch()
    sim = abi.OrcaSim.for_scene(batch.scenes[0])  # max_scenes 0
    with pytest.raises(abi.OrcaError) as e:
        sim.set_batch(batch)
    assert e.value.status == abi.ORCA_ERR_STATE
    sim2 = abi.OrcaSim(max_agents=batch.n, max_neighbors=8, neighbor_dist=10.0, dt=0.1, max_scenes=20)
    with pytest.raises(abi.OrcaError) as e:  # a scene asks for more neighbours than the context holds
        sim2.set_batch(batch)
    assert e.value.status == abi.ORCA_ERR_ARG
    sim3 = abi.OrcaSim(max_agents=batch.n, max_neighbors=20, neighbor_dist=10.0, dt=0.1, max_scenes=3)
    with pytest.raises(abi.OrcaError) as e:
        sim3.set_batch(batch)
    assert e.value.status == abi.ORCA_ERR_CAPACITY
