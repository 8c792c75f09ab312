"""Cell-size autotuner for the ORCA step.

The neighbour search is exact for any grid cell edge, so the edge is a pure speed knob:
too coarse and each agent scans many candidates, too fine and it visits many empty
cells.  ``tune_cell_size`` times a few steps of the real crowd through the library's
per-phase profiling events (on the context's current state; the state is restored
afterwards) for a set of edges expressed in units of the expected k-th neighbour
distance, and returns the fastest.  Results are cached in a JSON file keyed by
(agent-count bucket, density bucket, k).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import abi

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "orca_gb300_autotune.json")
# candidate edges, in units of the expected k-th neighbour distance sqrt(k / (pi rho))
FACTORS = (0.6, 0.8, 1.0, 1.2, 1.5, 2.0, 2.5)


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


def tune_cell_size(sim: "abi.OrcaSim", scene, steps: int = 6, factors=FACTORS,
                   cache_path: str | None = CACHE, use_cache: bool = True) -> dict:
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
    for f in factors:
        s = float(np.float32(f * rk))
        abi.orca_set_cell_size(sim.ctx, s)
        sim.set_scene(scene)
        sim.step(2)  # capture + warm up
        ms = []
        for _ in range(steps):
            sim.step(1)
            ms.append(float(abi.orca_profile_read(sim.ctx).sum()))
        timings[s] = float(np.median(ms))
    abi.orca_profile(sim.ctx, False)
    best = min(timings, key=timings.get)
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
