"""Multi-process host logic with torch.distributed over gloo (world_size 2, CPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1908_10107_gb300 import multigpu, scenarios as S


def test_shard_scenes_balanced_and_complete():
    counts = [s.n for s in S.batched().scenes]
    for world in (1, 2, 3, 4, 8):
        parts = multigpu.shard_scenes(counts, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(counts)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        loads = [sum(counts[a:b]) for a, b in parts]
        assert sum(loads) == sum(counts)
        assert max(loads) - min(loads) <= 2 * max(counts)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = [s.n for s in S.batched(n_scenes=40, seed=3).scenes]
    lo, hi = multigpu.shard_scenes(counts, world)[rank]
    units = float(sum(counts[lo:hi]))
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    value, mx = multigpu.job_throughput(units, ms, dist, device="cpu")
    dist.barrier()
    out[rank] = (lo, hi, value, mx)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    counts = [s.n for s in S.batched(n_scenes=40, seed=3).scenes]
    (a0, b0, v0, m0), (a1, b1, v1, m1) = out[0], out[1]
    assert (a0, b0, a1, b1)[0] == 0 and b0 == a1 and b1 == len(counts)
    assert m0 == m1 == 15.0
    assert v0 == v1 == pytest.approx(sum(counts) / 15e-3)
