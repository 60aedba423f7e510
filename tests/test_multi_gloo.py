"""Multi-rank host logic on CPU: two gloo ranks (127.0.0.1).

A single graph runs as replicas (the slowest rank's time, every rank's
work); a batch is split by arc count.  These tests run the rank logic the
benchmark uses, without a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2603_11645_gb300 import graphs, multi  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # replicas: each rank "measured" a different time; all see the max
        t = multi.max_over_ranks(10.0 + 5.0 * rank)
        rate = multi.whole_job_rate(1000.0, world, t / 1e3)
        # batch split: every rank computes the same split on its own
        b = graphs.workload_batch(G=64, seed=4)
        shards = multi.lpt_shards([g.A for g in b.graphs], world)
        mine = shards[rank]
        sub = graphs.pack_batch([b.graphs[i] for i in mine])
        tot = torch.tensor([float(sub.m), float(len(mine))], dtype=torch.float64)
        dist.all_reduce(tot)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, t, rate, tot.tolist(), gathered, b.m, b.G))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_batch_split():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, tot, gathered, m_all, G in out:
        assert t == 15.0                                   # the slowest rank's time
        assert rate == pytest.approx(1000.0 * 2 / 0.015)   # all ranks' units / that time
        assert tot == [float(m_all), float(G)]             # the shards cover the batch once
        flat = sorted(i for s in gathered for i in s)
        assert flat == list(range(G))                      # disjoint and complete
        assert gathered == out[0][4]                       # the same split on every rank


def test_lpt_split_is_balanced_and_deterministic():
    rng = np.random.default_rng(3)
    w = rng.integers(1, 1000, size=500)
    for world in (1, 2, 3, 8):
        s = multi.lpt_shards(w, world)
        assert s == multi.lpt_shards(w, world)
        assert sorted(i for x in s for i in x) == list(range(500))
        loads = [int(w[x].sum()) for x in s]
        # greedy LPT: no rank exceeds the mean by more than the heaviest item
        assert max(loads) <= w.sum() / world + w.max()


def test_single_process_needs_no_group():
    assert multi.max_over_ranks(3.5) == 3.5
    assert multi.whole_job_rate(10.0, 1, 2.0) == 5.0
