"""Host-side logic for several GPUs, one process per GPU.

A single graph does not shard (every contraction round exchanges labels and
list ranking chases pointers across the whole successor array), so N GPUs run
N independent replicas.  A batch of graphs does shard: the graphs are split
by arc count with the greedy longest-processing-time rule and each rank builds
its share with one rst_build_batch call; no data-path collective is needed,
only a max over ranks of the measured time.
"""
from __future__ import annotations

import numpy as np


def lpt_shards(weights, world: int) -> list[list[int]]:
    """Indices of `weights` split into `world` lists: heaviest first, each to
    the currently lightest rank (ties: the lower rank).  Deterministic, so
    every rank computes the same split without communicating."""
    w = np.asarray(weights, dtype=np.float64)
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    loads = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        out[r].append(i)
        loads[r] += w[i]
    for lst in out:
        lst.sort()
    return out


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks of the default process group (the
    slowest rank decides a parallel step's time); `value` itself when no
    group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Throughput of N replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / max_seconds
