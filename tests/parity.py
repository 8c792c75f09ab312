"""Helpers for GPU-vs-oracle parity: run steps through the C ABI, run the oracle on the
same FP32 state, and compare.

The bar (the same in every GPU test):
  * cell of every agent and the grid: bit-exact;
  * neighbour lists (indices and order): bit-exact;
  * velocity: |v_gpu - v_oracle| <= VEL_TOL m/s per agent (FP32 against FP64), except for
    agents the oracle tags as ill-conditioned: a discontinuous half-plane decision taken
    within a relative MARGIN of its threshold, or an LP whose answer moves by more than
    SENS_MAX under FP32-rounding-sized perturbations of its half-planes (there FP32 and
    FP64 may legitimately differ).  The agents the tags excuse -- tagged AND outside
    VEL_TOL -- may be at most TAGGED_MAX of the agents compared, rounded up to a whole
    agent (the gate's reading of "tagged agents are excluded and must be at most 0.1%":
    a tagged agent that meets the bar is not excluded from anything).  However many
    agents a faulty tagger marked, it could excuse no more than that;
  * position: every agent moves by its own velocity, |p_gpu - (p + v_gpu dt)| <= 2 ulp, and
    |p_gpu - p_oracle| <= max(VEL_TOL, |v_gpu - v_oracle|) * dt + 2 ulp(|p|) (FP32 storage
    of p): a tagged agent's position may differ only by its velocity's difference.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_1908_10107_gb300 import abi

VEL_TOL = 1e-4
MARGIN = 1e-4
SENS_MAX = 0.5 * VEL_TOL
TAGGED_MAX = 1e-3


def tagged_cap(rows: int) -> int:
    """Most agents of ``rows`` the tags may excuse from the velocity bar: 0.1%, rounded up."""
    return max(1, math.ceil(TAGGED_MAX * rows))


def make_sim(scene, flags=abi.ORCA_FLAG_RECORD, cell_size=0.0, max_cells=0, max_agents=None):
    return abi.OrcaSim(max_agents=max_agents or max(scene.n, 1),
                       max_neighbors=scene.max_neighbors, neighbor_dist=scene.neighbor_dist,
                       dt=scene.dt, cell_size=cell_size, max_cells=max_cells, flags=flags)


def effective_cell_size(scene, cell_size):
    return cell_size if cell_size > 0 else scene.neighbor_dist * 0.25


def effective_max_cells(n, max_cells):
    return max_cells if max_cells > 0 else min(max(4 * n, 65536), 1 << 30)


def compare_step(scene, gpu_pos, gpu_vel, gpu_nbr, gpu_cells=None, gpu_grid=None,
                 cell_size=0.0, max_cells=0, subset=None, gpu_obst=None):
    """Oracle one step from ``scene``'s FP32 state; compare with the GPU's results (rows of
    agents ``subset`` if given).  Returns a report dict; raises AssertionError on failure."""
    n = scene.n
    rows = np.arange(n) if subset is None else np.asarray(subset)
    if gpu_grid is not None:
        gf, gi = oracle.grid(scene.pos, effective_cell_size(scene, cell_size),
                             effective_max_cells(n, max_cells))
        np.testing.assert_array_equal(gpu_grid[0], gf, err_msg="grid floats differ")
        np.testing.assert_array_equal(gpu_grid[1], gi, err_msg="grid dims differ")
        if gpu_cells is not None:
            want = oracle.cells(scene.pos, gf, gi)
            np.testing.assert_array_equal(gpu_cells, want, err_msg="cells differ")
    ref = oracle.step_scene(scene, knn_mode=1, subset=None if subset is None else rows,
                            sensitivity=True)
    np.testing.assert_array_equal(gpu_nbr[rows], ref["nbr"], err_msg="neighbour lists differ")
    if gpu_obst is not None:
        ko = ref["obst"].shape[1]
        np.testing.assert_array_equal(gpu_obst[rows][:, :ko], ref["obst"],
                                      err_msg="obstacle neighbours differ")
    dv = np.abs(gpu_vel[rows].astype(np.float64) - ref["vel"]).max(axis=1)
    tagged = (ref["margin"] < MARGIN) | (ref["sens"] > SENS_MAX)
    bad = dv > VEL_TOL
    untagged_bad = np.flatnonzero(bad & ~tagged)
    tagged_bad = int((bad & tagged).sum())
    rep = dict(rows=len(rows), max_dv_untagged=float(dv[~tagged].max(initial=0.0)),
               tagged=int(tagged.sum()), tagged_bad=tagged_bad, lp3=int(ref["lp3"].sum()),
               max_dv=float(dv.max(initial=0.0)))
    assert untagged_bad.size == 0, (
        f"velocity mismatch on {untagged_bad.size} well-conditioned agents; first rows "
        f"{rows[untagged_bad[:5]].tolist()} dv={dv[untagged_bad[:5]].tolist()} report={rep}")
    assert tagged_bad <= tagged_cap(len(rows)), f"too many agents excused by their tags {rep}"
    p = gpu_pos[rows].astype(np.float64)
    dt = np.float64(np.float32(scene.dt))
    ulp2 = 2.0 * np.spacing(np.abs(p).astype(np.float32)).astype(np.float64)
    own = np.asarray(scene.pos, np.float32)[rows].astype(np.float64) + \
        gpu_vel[rows].astype(np.float64) * dt
    ok_own = np.abs(p - own) <= ulp2
    assert ok_own.all(), f"{int((~ok_own).any(1).sum())} agents did not move by their velocity {rep}"
    tolp = np.maximum(VEL_TOL, dv)[:, None] * dt + ulp2
    okp = np.abs(p - ref["pos"]) <= tolp
    assert okp.all(), f"position mismatch on {int((~okp).any(1).sum())} agents {rep}"
    return rep


def gpu_step_and_compare(scene, steps_before=0, cell_size=0.0, max_cells=0, sim=None,
                         subset=None):
    """Load ``scene``; run ``steps_before`` steps; then one recorded step compared with the
    oracle started from the GPU's FP32 state at that point."""
    own = sim is None
    sim = sim or make_sim(scene, cell_size=cell_size, max_cells=max_cells)
    sim.set_scene(scene)
    st = scene.copy()
    if steps_before:
        # continue from the GPU's own (cell-permuted) layout; the oracle starts from the
        # read-out FP32 state
        sim.step(steps_before)
        pos, vel = sim.get_state()
        st.pos, st.vel = pos, vel
    sim.step(1)
    pos, vel = sim.get_state()
    nbr = sim.get_neighbors()
    cells, gf, gi = sim.get_cells()
    obst = sim.get_obstacle_neighbors() if getattr(st, "obstacles", None) is not None else None
    rep = compare_step(st, pos, vel, nbr, cells, (gf, gi), cell_size, max_cells, subset, obst)
    if own:
        sim.close()
    return rep
