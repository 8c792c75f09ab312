"""Host logic for running on several GPUs, one process per GPU.

The ORCA step has no exchange between independent crowds, so multi-GPU runs need no data
collective:
  * a single crowd runs as identical replicas (one per rank);
  * a batch of independent scenes is split across ranks by agent count, each rank
    advancing its own scenes (weak scaling).
The only collectives are the timing ones: a barrier around the timed region and the
maximum of the ranks' device times, from which the whole-job throughput follows.
"""
from __future__ import annotations

import numpy as np


def shard_scenes(counts, world: int):
    """Split scenes (agent counts) into `world` contiguous groups of nearly equal agents.
    Returns a list of (first, last+1) scene ranges; deterministic, same on every rank."""
    counts = np.asarray(counts, dtype=np.int64)
    total = int(counts.sum())
    bounds = [0]
    cum = np.cumsum(counts)
    for r in range(1, world):
        target = total * r / world
        # first scene boundary at or after the target, kept non-decreasing
        b = int(np.searchsorted(cum, target, side="left")) + 1
        bounds.append(max(min(b, len(counts)), bounds[-1]))
    bounds.append(len(counts))
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def job_throughput(local_units: float, local_ms: float, dist=None, device=None) -> tuple:
    """Whole-job throughput: sum of the units every rank processed over the slowest rank's
    time.  Returns (units per second, max ms)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_units / (local_ms * 1e-3), local_ms
    import torch
    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t[1:].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tot.item()) / (float(mx.item()) * 1e-3), float(mx.item())
