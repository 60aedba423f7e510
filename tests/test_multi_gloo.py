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
        # the rank's packed shard holds exactly its graphs: the oracle's tree
        # of every graph read back from the packed arrays equals the one of
        # the original graph
        import oracle
        for j, gi in enumerate(mine):
            g = b.graphs[gi]
            o, c = sub.graph_offsets(j), sub.graph_cols(j)
            assert int(sub.roots[j]) == g.root
            assert np.array_equal(oracle.rst(g.n, o, c, int(sub.roots[j])),
                                  oracle.rst(g.n, g.offsets, g.cols, g.root))
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


def test_bench_starts_one_rank_per_gpu():
    """`bench.py --gpus 2` without a launcher starts two ranks itself; rank 0
    alone prints the JSON line, with n_gpus = 2 (the reference arm runs on
    the host, so this works without a GPU)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    import bench
    cmd = bench.launch_command(["--gpus", "2"], 2, 12345)
    assert cmd[:3] == [sys.executable, "-m", "torch.distributed.run"]
    assert "--nproc-per-node=2" in cmd and "127.0.0.1" in cmd and cmd[-2:] == ["--gpus", "2"]
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["impl"] == "reference" and line["value"] > 0
