"""The ORCA_CHECKS build: the same kernels with device-side index checks.

compute-sanitizer is not available here, so the library has a build of its own that tests
every index it computes from data (cell-table positions, candidate and neighbour slots,
agent ids, cell keys) before using it and latches ORCA_ERR_BOUNDS instead of accessing out
of range.  On consistent inputs no check may fire, and the checked build must give bitwise
the results of the ordinary one (and so pass the oracle parity bar).
"""
import numpy as np
import pytest

from paper_1908_10107_gb300 import abi
from paper_1908_10107_gb300 import scenarios as S

import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checks_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_10107_gb300 import build
    build.build()
    return build.build(checks=True)


def _run(scene, steps, cell_size=0.0):
    sim = parity.make_sim(scene, cell_size=cell_size)
    sim.set_scene(scene)
    sim.step(steps)
    abi.orca_sync(sim.ctx)  # raises on a latched device error (ORCA_ERR_BOUNDS among them)
    pos, vel = sim.get_state()
    nbr = sim.get_neighbors()
    search = sim.search_counters()
    sim.close()
    return pos, vel, nbr, search


@pytest.mark.parametrize("scene,steps,cell", [
    (S.jitter_velocities(S.bidirectional(8190, seed=61), 61), 12, 0.0),
    (S.dense(6000, seed=62, max_neighbors=20), 6, 0.0),
    (S.circle_swap(1024), 30, 0.05),
    (S.two_way_crossing(2500, heterogeneous=True), 40, 0.0),
])
def test_checked_build_fires_no_check_and_matches_bitwise(checks_lib, scene, steps, cell):
    want = _run(scene, steps, cell)
    with abi.use_library(checks_lib):
        got = _run(scene, steps, cell)
    for a, b in zip(got[:3], want[:3]):
        np.testing.assert_array_equal(a, b)
    # the rows a search scans depend on when its bound tightens, and so on the order of the
    # agents inside a cell, which varies between runs; the passes and starts do not
    for key in ("extra_passes", "unpredicted"):
        assert got[3][key] == want[3][key]


def test_checked_build_passes_the_parity_bar(checks_lib):
    sc = S.jitter_velocities(S.bidirectional(4099, seed=63), 63)
    with abi.use_library(checks_lib):
        rep = parity.gpu_step_and_compare(sc, steps_before=5)
    assert rep["rows"] == sc.n


def _grads(torch, sc, W, T, C):
    sim = abi.OrcaSim.for_scene(sc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in sc.arrays()]
    sim.set_agents(*dev)
    nbytes = abi.orca_rollout_workspace_size(sim.ctx, T, C)
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    ws = raw[off: off + nbytes]
    traj = torch.empty((T, sc.n, 2), device="cuda")
    abi.orca_rollout_forward(sim.ctx, T, C, traj, ws)
    g = [torch.empty(sc.n, device="cuda") for _ in range(3)]
    gp0 = torch.empty((sc.n, 2), device="cuda")
    gv0 = torch.empty((sc.n, 2), device="cuda")
    abi.orca_rollout_backward(sim.ctx, torch.from_numpy(W).float().cuda(), g[0], g[1], g[2], gp0, gv0, ws)
    abi.orca_sync(sim.ctx)
    out = [x.cpu().numpy() for x in (traj, *g, gp0, gv0)]
    sim.close()
    return out


@pytest.mark.parametrize("C", [0, 4])
def test_checked_build_adjoint_overflow_scan_matches_bitwise(checks_lib, C):
    """The checked build gives each agent two places for the entries it receives, so most
    agents of a crowd take their entries from the scan of all agents' entries: the sums
    meet the entries in the same order and must agree bit for bit with the lists."""
    import torch
    sc = S.jitter_velocities(S.bidirectional(2500, seed=64), 64)
    W = np.random.default_rng(5).standard_normal((9, sc.n, 2))
    want = _grads(torch, sc, W, 9, C)
    with abi.use_library(checks_lib):
        got = _grads(torch, sc, W, 9, C)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)
    assert np.abs(want[2]).max() > 0
