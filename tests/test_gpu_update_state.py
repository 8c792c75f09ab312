"""orca_update_state: new positions / velocities for the current agents, with parameters,
memory order and search-radius predictions kept."""
import numpy as np
import pytest

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


def test_writing_back_the_read_state_changes_nothing():
    sc = S.jitter_velocities(S.bidirectional(6000, seed=51), 51)
    a = parity.make_sim(sc, flags=0)
    b = parity.make_sim(sc, flags=0)
    a.set_scene(sc)
    b.set_scene(sc)
    a.step(5)
    b.step(5)
    for _ in range(10):
        pos, vel = b.get_state()
        b.update_state(pos, vel)
        b.step(1)
        a.step(1)
    pa, va = a.get_state()
    pb, vb = b.get_state()
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)
    a.close()
    b.close()


@pytest.mark.parametrize("device", [False, True])
def test_an_edited_state_steps_like_the_oracle(device):
    import torch
    sc = S.jitter_velocities(S.bidirectional(4000, seed=52), 52)
    sim = parity.make_sim(sc)
    sim.set_scene(sc)
    sim.step(7)  # the memory order is now the cell order, not the agent order
    pos, vel = sim.get_state()
    rng = np.random.default_rng(52)
    pos2 = (pos + rng.normal(0, 0.05, pos.shape)).astype(np.float32)
    vel2 = (vel + rng.normal(0, 0.3, vel.shape)).astype(np.float32)
    if device:
        sim.update_state(torch.from_numpy(pos2).cuda(), torch.from_numpy(vel2).cuda())
    else:
        sim.update_state(pos2, vel2)
    got = sim.get_state()
    np.testing.assert_array_equal(got[0], pos2)
    np.testing.assert_array_equal(got[1], vel2)
    st = sc.copy()
    st.pos, st.vel = pos2, vel2
    sim.step(1)
    p3, v3 = sim.get_state()
    nbr = sim.get_neighbors()
    cells, gf, gi = sim.get_cells()
    parity.compare_step(st, p3, v3, nbr, cells, (gf, gi))
    sim.close()


def test_one_half_at_a_time_and_in_a_batch():
    sc = S.bidirectional(3000, seed=53)
    sim = parity.make_sim(sc, flags=0)
    sim.set_scene(sc)
    sim.step(3)
    pos, vel = sim.get_state()
    sim.update_state(vel=np.zeros_like(vel))
    p1, v1 = sim.get_state()
    np.testing.assert_array_equal(p1, pos)
    assert not v1.any()
    sim.update_state(pos=pos + np.float32(1.0))
    p2, v2 = sim.get_state()
    np.testing.assert_array_equal(p2, pos + np.float32(1.0))
    assert not v2.any()
    sim.close()
    batch = S.Batch([S.bidirectional(700, seed=54), S.two_way_crossing(500, seed=55)])
    bs = abi.OrcaSim.for_batch(batch)
    bs.set_batch(batch)
    bs.step(4)
    pos, vel = bs.get_state()
    bs.update_state(pos, -vel)
    p, v = bs.get_state()
    np.testing.assert_array_equal(p, pos)
    np.testing.assert_array_equal(v, -vel)
    bs.close()


def test_pinned_host_arrays_take_the_direct_path_and_agree():
    # pinned host memory is read and written by the kernels over the CPU-GPU link; pageable
    # memory goes through staging copies: both give the same state
    import torch
    sc = S.jitter_velocities(S.bidirectional(5000, seed=56), 56)
    sim = parity.make_sim(sc, flags=0)
    sim.set_scene(sc)
    sim.step(6)
    pos, vel = sim.get_state()
    ppos = torch.empty(pos.shape, dtype=torch.float32).pin_memory()
    pvel = torch.empty(vel.shape, dtype=torch.float32).pin_memory()
    abi.orca_get_state(sim.ctx, ppos, pvel)
    np.testing.assert_array_equal(ppos.numpy(), pos)
    np.testing.assert_array_equal(pvel.numpy(), vel)
    rng = np.random.default_rng(56)
    ppos.copy_(torch.from_numpy((pos + rng.normal(0, 0.02, pos.shape)).astype(np.float32)))
    pvel.copy_(torch.from_numpy((-vel).astype(np.float32)))
    sim.update_state(ppos, pvel)
    got = sim.get_state()
    np.testing.assert_array_equal(got[0], ppos.numpy())
    np.testing.assert_array_equal(got[1], pvel.numpy())
    sim.update_state(pos=None, vel=pvel.numpy())  # a numpy view of pinned memory
    np.testing.assert_array_equal(sim.get_state()[1], pvel.numpy())
    sim.close()


def test_pinned_transfers_across_reorders_odd_counts_and_unaligned_views():
    # the agent -> slot map is the last reorder's after a step, built afresh after a load or
    # a removal; an odd count leaves one agent outside the 16-byte pairs; a view that does
    # not start on 16 bytes takes the staging path
    import torch
    sc = S.jitter_velocities(S.two_way_crossing(5001, seed=57), 57)
    sim = parity.make_sim(sc, flags=0)
    sim.set_scene(sc)
    n = sc.n
    assert n % 2 == 1
    pin = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    pin_v = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    wide = torch.empty((n + 1, 2), dtype=torch.float32).pin_memory()
    odd = wide[1:]  # pinned, but 8 bytes past a 16-byte boundary

    def check():
        pos, vel = sim.get_state()  # pageable: staging copies
        abi.orca_get_state(sim.ctx, pin, pin_v)
        np.testing.assert_array_equal(pin.numpy(), pos)
        np.testing.assert_array_equal(pin_v.numpy(), vel)
        abi.orca_get_state(sim.ctx, odd, None)
        np.testing.assert_array_equal(odd.numpy(), pos)
        return pos, vel

    check()  # no step yet: agent order, map built from the ids
    sim.step(9)
    pos, vel = check()  # map from the last reorder
    rng = np.random.default_rng(57)
    new_pos = (pos + rng.normal(0, 0.01, pos.shape)).astype(np.float32)
    odd.copy_(torch.from_numpy(new_pos))
    sim.update_state(odd, None)  # staging path
    np.testing.assert_array_equal(sim.get_state()[0], new_pos)
    pin_v.copy_(torch.from_numpy((0.5 * vel).astype(np.float32)))
    sim.update_state(None, pin_v)  # direct path, map from the last reorder
    np.testing.assert_array_equal(sim.get_state()[1], (0.5 * vel).astype(np.float32))
    # after a removal the survivors are renumbered and the map is rebuilt
    sc2 = sc.copy()
    sc2.pos, sc2.vel = sim.get_state()
    sc2.goal = sc2.goal.copy()
    sc2.goal[::3] = sc2.pos[::3]
    sim.set_scene(sc2)
    sim.step(1)
    m, kept = sim.remove_arrived()
    assert 0 < m < n
    pos_m, vel_m = sim.get_state()
    p_m = torch.empty((m, 2), dtype=torch.float32).pin_memory()
    abi.orca_get_state(sim.ctx, p_m, None)
    np.testing.assert_array_equal(p_m.numpy(), pos_m)
    p_m.copy_(torch.from_numpy((pos_m + np.float32(0.25)).astype(np.float32)))
    sim.update_state(p_m, None)
    np.testing.assert_array_equal(sim.get_state()[0], pos_m + np.float32(0.25))
    sim.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_step_host_is_write_step_read(pinned):
    # the fused call equals orca_update_state + orca_step + orca_get_state, bitwise, also
    # with the output written over the input
    import torch
    sc = S.jitter_velocities(S.bidirectional(4001, seed=58), 58)
    a = parity.make_sim(sc, flags=0)
    b = parity.make_sim(sc, flags=0)
    a.set_scene(sc)
    b.set_scene(sc)
    a.step(4)
    b.step(4)

    def buf(x):
        if not pinned:
            return np.ascontiguousarray(x)
        t = torch.empty(x.shape, dtype=torch.float32).pin_memory()
        t.copy_(torch.from_numpy(np.ascontiguousarray(x)))
        return t.numpy()

    pos, vel = a.get_state()
    io_pos, io_vel = buf(pos), buf(vel)
    for it in range(5):
        nsteps = 2 if it % 2 else 1
        # a: separate calls; b: one fused call writing its result over its input
        pa, va = a.get_state()
        a.update_state(pa, va)
        a.step(nsteps)
        want = a.get_state()
        b.step_host(io_pos, io_vel, nsteps, io_pos, io_vel)
        np.testing.assert_array_equal(io_pos, want[0])
        np.testing.assert_array_equal(io_vel, want[1])
    # nothing in, nothing stepped: a plain read
    out = buf(np.zeros_like(pos))
    b.step_host(None, None, 0, out, None)
    np.testing.assert_array_equal(out, want[0])
    a.close()
    b.close()
