"""Autotuner for the ORCA step: grid cell edge and launch shape.

The neighbour search is exact for any grid cell edge, so the edge is a pure speed knob:
too coarse and each agent scans many candidates, too fine and it visits many empty
cells.  ``tune_cell_size`` times a few steps of the real crowd through the library's
per-phase profiling events (on the context's current state; the state is restored
afterwards) for a set of edges expressed in units of the expected k-th neighbour
distance, re-times the two fastest with twice the steps, and returns the faster.  A
``between`` callable, run before every timed step, lets a caller reproduce its own
conditions (an L2 flush, say) while tuning.  Results are cached in a JSON file keyed by
(agent-count bucket, density bucket, k).

``tune_launch`` then tries the per-agent kernel's launch shapes (64 or 128 threads per CTA)
and LP modes (one lane per solve, warp work units); ``tune_batch`` does both for a batch of
scenes, where each scene's edge is a common factor times its own expected k-th neighbour
distance.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import abi

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "orca_gb300_autotune.json")
# candidate edges, in units of the expected k-th neighbour distance sqrt(k / (pi rho)).
# Measured on the 524,288-agent flow, edges between 0.8 and 1.5 of that distance lie
# within 1% of each other and the extremes 0.6 and 2.5 cost 6-11% more, so the sweep
# keeps the band where the optimum has been found on every workload measured.
FACTORS = (0.8, 1.0, 1.2, 1.5, 2.0)


def expected_kth_distance(pos: np.ndarray, k: int) -> float:
    """sqrt(k / (pi * rho)) with rho the density over the occupied 8 m x 8 m tiles."""
    p = np.asarray(pos, np.float64).reshape(-1, 2)
    tiles = np.unique(np.floor(p / 8.0).astype(np.int64), axis=0).shape[0]
    rho = p.shape[0] / max(tiles * 64.0, 1e-9)
    return math.sqrt(k / (math.pi * rho))


def _key(n: int, rk: float, k: int) -> str:
    return f"n2^{int(round(math.log2(max(n, 1))))}-rk{rk:.2g}-k{k}"


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


# timed steps per candidate, after WARM untimed ones (the first steps after a reload are
# not typical: a crowd that starts at rest turns to its preferred velocities in step 1)
STEPS, WARM = 16, 8


def tune_cell_size(sim: "abi.OrcaSim", scene, steps: int = STEPS, factors=FACTORS,
                   cache_path: str | None = CACHE, use_cache: bool = True,
                   between=None) -> dict:
    """Pick the fastest cell edge for ``scene`` on ``sim`` (which must hold the scene).

    Returns {"cell_size": s, "timings_ms": {s: ms}, "kth_distance": rk, "cached": bool} and
    leaves ``sim`` with that edge and the scene's state reloaded."""
    rk = expected_kth_distance(scene.pos, scene.max_neighbors)
    key = _key(scene.n, rk, scene.max_neighbors)
    cache = _load_cache(cache_path) if (cache_path and use_cache) else {}
    if key in cache:
        s = float(cache[key]["cell_size"])
        abi.orca_set_cell_size(sim.ctx, s)
        sim.set_scene(scene)
        return {"cell_size": s, "timings_ms": cache[key].get("timings_ms", {}),
                "kth_distance": rk, "cached": True}
    timings = {}
    abi.orca_profile(sim.ctx, True)

    def with_edge(s):
        def reload():
            abi.orca_set_cell_size(sim.ctx, s)
            sim.set_scene(scene)
        return reload

    for f in factors:
        s = float(np.float32(f * rk))
        timings[s] = _time_steps(sim, with_edge(s), steps, between)
    best = _refine(sim, timings, with_edge, steps, between)
    abi.orca_profile(sim.ctx, False)
    abi.orca_set_cell_size(sim.ctx, best)
    sim.set_scene(scene)
    if cache_path:
        cache = _load_cache(cache_path)
        cache[key] = {"cell_size": best, "timings_ms": {str(k): v for k, v in timings.items()}}
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return {"cell_size": best, "timings_ms": timings, "kth_distance": rk, "cached": False}


# Launch shapes tried: (threads per CTA, LP mode).  256-thread CTAs ran slower than these
# on every workload measured (the 524,288-agent flow, the dense crowd at k = 10 and 20, the
# 256-scene batch: 5-30%), so they are not tried; they stay available through
# orca_set_launch.  One lane per solve wins at k = 10, warp work units at k = 20, and the
# agent split (four lanes per agent) in crowds of a few thousand agents; a batch never
# runs the split (its persistent kernel keeps one lane per agent).
SHAPES = ((64, 1), (128, 1), (64, 32), (128, 32), (64, 4))
BATCH_SHAPES = ((64, 1), (128, 1), (64, 32), (128, 32))


def _time_steps(sim, reload, steps, between=None):
    """Median device time of ``steps`` single steps (profiling events on) after a reload
    and WARM untimed steps (graph capture, warm-up)."""
    reload()
    sim.step(WARM)
    ms = []
    for _ in range(steps):
        if between is not None:
            between()
        sim.step(1)
        ms.append(float(abi.orca_profile_read(sim.ctx).sum()))
    return float(np.median(ms))


def _refine(sim, timings, make_reload, steps, between):
    """The faster of the two best candidates in ``timings``, re-timed in alternation with
    twice the steps (a single sweep's ranking of near-equal candidates is noise)."""
    ranked = sorted(timings, key=timings.get)
    if len(ranked) < 2:
        return ranked[0]
    acc = {c: [] for c in ranked[:2]}
    for _ in range(2):
        for c in ranked[:2]:
            acc[c].append(_time_steps(sim, make_reload(c), steps, between))
    return min(acc, key=lambda c: float(np.mean(acc[c])))


def tune_launch(sim: "abi.OrcaSim", reload, steps: int = STEPS, shapes=SHAPES,
                between=None) -> dict:
    """Fastest (threads per CTA, LP3 lanes) for the crowd that ``reload()`` loads into
    ``sim``; leaves ``sim`` set to it and reloaded."""
    abi.orca_profile(sim.ctx, True)

    def with_shape(shape):
        def go():
            abi.orca_set_launch(sim.ctx, *shape)
            reload()
        return go

    timings = {}
    for shape in shapes:
        timings[shape] = _time_steps(sim, with_shape(shape), steps, between)
    best = _refine(sim, timings, with_shape, steps, between)
    abi.orca_profile(sim.ctx, False)
    abi.orca_set_launch(sim.ctx, *best)
    reload()
    return {"shape": best, "timings_ms": {f"{a}x{b}": v for (a, b), v in timings.items()}}


def batch_cell_sizes(batch, factor: float):
    return [float(np.float32(factor * expected_kth_distance(sc.pos, sc.max_neighbors)))
            if sc.n > 1 else 0.0 for sc in batch.scenes]


def set_batch_cells(sim, batch, cells):
    params = [(sc.n, sc.max_neighbors, sc.neighbor_dist, sc.dt, cs)
              for sc, cs in zip(batch.scenes, cells)]
    sim.n_scenes = len(batch.scenes)
    abi.orca_set_scenes(sim.ctx, params, *batch.arrays())


def tune_batch(sim: "abi.OrcaSim", batch, steps: int = STEPS, factors=FACTORS, shapes=BATCH_SHAPES,
               between=None) -> dict:
    """Cell-edge factor (common to all scenes, times each scene's expected k-th neighbour
    distance) and launch shape for a batch; leaves ``sim`` tuned with the batch loaded."""
    abi.orca_profile(sim.ctx, True)

    def with_factor(f):
        cells = batch_cell_sizes(batch, f)
        return lambda: set_batch_cells(sim, batch, cells)

    ftimes = {f: _time_steps(sim, with_factor(f), steps, between) for f in factors}
    best_f = _refine(sim, ftimes, with_factor, steps, between)
    cells = batch_cell_sizes(batch, best_f)
    shape = tune_launch(sim, lambda: set_batch_cells(sim, batch, cells), steps, shapes, between)
    return {"factor": best_f, "factor_timings_ms": ftimes, "cell_sizes": cells, **shape}
