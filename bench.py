#!/usr/bin/env python3
"""Benchmark: rooted-spanning-tree build throughput on one GB300 (edges/s = m/time).

Headline: CC+Euler (hook/compress connectivity + Euler-tour rooting) on the
high-diameter workload, a 4096 x 4096 4-neighbour grid with seed-permuted ids
and a seeded random root (16,777,216 vertices, 33,546,240 undirected edges,
int32 CSR).  One step = one rst_build(RST_CC_EULER) over the resident graph.
Beside it: the library's own level-synchronous GPU BFS on the same graph, the
per-kernel roofline of the dominant kernel, the end-to-end number through the
C ABI with host buffers, and the CPU oracle timed on the host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 the script starts N ranks itself (torchrun, one process per
GPU) unless a launcher already did.  Every rank builds the same graph on its
own GPU: the single-graph path does not shard, so ranks are replicas
("scaling": "weak"); the batch of graphs is split by arc count.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RST build edges/s (m/time) per graph family vs own GPU BFS; selector regret %"
WORKLOAD = ("grid 4096x4096 4-neighbour, ids permuted by seed 2, seeded random root, "
            "int32 CSR (16,777,216 vertices, 33,546,240 undirected edges)")
L2_BYTES = 129 * 1024 * 1024


# ----------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_bytes(name, n, A, st, o):
    """Algorithmic bytes per launch: every element a kernel must read or write,
    counted once (random accesses are not charged their sector size).
    N = tree arcs list-ranked (after leaf pruning), T = tree edges."""
    T = st["T"]
    N = st["lr_n"]
    K = N // 2  # tree edges that are toured
    c1, E2 = st["c1"], st["E2"]
    models = {
        # offsets, the first entries of every row, P and J, a 32-byte row record
        "k_r1_choose": (n + 1) * o + 4 * n + 8 * n + 32 * n,
        # P, J, P written per vertex; per non-root the used part of the chosen
        # neighbour's row record (start, degree and its row's entries, at most
        # six) and a 16-byte tree-edge record
        "k_r1_resolve": 16 * n + (n - c1) * (8 + 4 * min(A / max(n, 1), 6) + 16) + 4 * n,
        # J and P per vertex, its label written, the root bitmap and prefix
        # read once, the minimum vertex of every round-1 component written
        "k_r1_label": 12 * n + n // 4 + 4 * c1,
        "k_build_list": (n + 1) * o + 4 * A + 4 * n + 2 * A + 12 * E2,
        # offsets, the ranked tree bitmap at both row ends, the root bit, the
        # leaf flag written
        "k_run_flags": (n + 1) * o + 8 * n + n // 8 + n,
        # offsets read, the row-start bitmap written
        "k_row_starts": (n + 1) * o + A // 8,
        "k_prune_leaves": 16 * T + 2 * T + 4 * (T - K),
        # per toured edge: its record rewritten, both arcs' ranked words, the
        # row-start words after both arcs and a root bit, two successors
        "k_pairs_succ": 16 * T + K * (16 + 16 + 12 + 8),
        # successor read and packed 4-byte record written per element; per
        # splitter its start, next splitter and weight
        "k_lr_walk1": 8 * N + 12 * ((N + 15) // 16),
        "k_lr_final1": 4 * N + 4 * N + 4 * ((N + 15) // 16),
        "k_parent_from_rank": 16 * T + K * (8 + 4),
        # the same reading two packed first-level records and two splitter
        # positions per toured edge instead of two positions
        "k_parent_from_owner": 16 * T + K * (8 + 8 + 4),
    }
    return models.get(name)


def run_e2e_streamed(rst, g, off, col, par, off_h, col_h, dev, stream, steps, world):
    """The end-to-end rate of a stream of builds: the same pinned-host CSR
    copied in and the parents copied out every step, double-buffered so that
    step i+1's host-to-device copy (on a copy stream) runs while step i
    builds and step i's parents go back while step i+1 builds.  Every copy of
    every step is inside the timed region (first event before the first
    copy, last after the last parents arrive)."""
    import torch
    from paper_2603_11645_gb300 import multi
    steps = max(2, steps)
    cp_in = torch.cuda.Stream(dev)
    cp_out = torch.cuda.Stream(dev)
    offs = [torch.empty_like(off) for _ in range(2)]
    cols = [torch.empty_like(col) for _ in range(2)]
    pars = [torch.empty_like(par) for _ in range(2)]
    par_h = [torch.empty(g.n, dtype=torch.int32).pin_memory() for _ in range(2)]
    for b in range(2):  # untimed first copies into the fresh buffers
        offs[b].copy_(off_h, non_blocking=True)
        cols[b].copy_(col_h, non_blocking=True)
        par_h[b].copy_(par, non_blocking=True)
    ev = lambda: torch.cuda.Event()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    in_done = [ev() for _ in range(steps)]
    built = [ev() for _ in range(steps)]
    out_done = [ev() for _ in range(steps)]
    torch.cuda.synchronize(dev)
    e0.record(stream)
    cp_in.wait_event(e0)

    def copy_in(i):
        b = i % 2
        if i >= 2:
            cp_in.wait_event(built[i - 2])  # build i-2 has finished reading buffer b
        with torch.cuda.stream(cp_in):
            offs[b].copy_(off_h, non_blocking=True)
            cols[b].copy_(col_h, non_blocking=True)
        in_done[i].record(cp_in)

    copy_in(0)
    for i in range(steps):
        b = i % 2
        if i + 1 < steps:
            copy_in(i + 1)
        stream.wait_event(in_done[i])
        if i >= 2:
            stream.wait_event(out_done[i - 2])  # parents of step i-2 are out of buffer b
        rst.build(offs[b], cols[b], g.root, "cc_euler", out=pars[b])
        built[i].record(stream)
        cp_out.wait_event(built[i])
        with torch.cuda.stream(cp_out):
            par_h[b].copy_(pars[b], non_blocking=True)
        out_done[i].record(cp_out)
    stream.wait_event(out_done[steps - 1])
    stream.wait_event(out_done[steps - 2])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = multi.max_over_ranks(e0.elapsed_time(e1), dev)
    assert torch.equal(par_h[(steps - 1) % 2].to(dev), par)
    return {"value": multi.whole_job_rate(g.m * steps, world, ms / 1e3), "unit": "edges/s",
            "steps": steps, "h2d_bytes_per_step": int(g.offsets.nbytes + g.cols.nbytes),
            "d2h_bytes_per_step": int(4 * g.n),
            "schedule": "double-buffered stream of builds: step i+1's CSR copy in and step i-1's "
                        "parents copy out overlap step i's build"}


def step_bytes_model(n, A, T, o):
    """Algorithmic bytes of one whole CC+Euler step (the hot-path byte model):
    connectivity reads the offsets and every column once, gathers one 4-byte
    label per arc, reads and writes the labels and writes the tree edges
    (o(n+1) + 8A + 16n + 8T); the Euler stage moves about 60 bytes per tree
    arc (arc generation, one counting pass over key and value, next, succ,
    rank read and write, twin reads) plus 12 per vertex (60E + 12n, E = 2T)."""
    return o * (n + 1) + 8 * A + 16 * n + 8 * T + 60 * (2 * T) + 12 * n


def step_roofline(n, A, T, o, ms, peak):
    """The whole step against the byte model: bytes / time over the peak."""
    byts = step_bytes_model(n, A, T, o)
    achieved = byts / (ms / 1e3) / 1e9
    return {"bound": "hbm", "algorithmic_bytes": int(byts), "ms": round(ms, 4),
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "roof_ms": round(byts / (peak * 1e9) * 1e3, 4)}


def host_cpu():
    """Model name and logical core count of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":", 1)
                if len(k) == 2 and k[0].strip() in ("model name", "Model name", "CPU part", "Hardware"):
                    model = model or k[1].strip()
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def _function_source(path, name):
    """Text of the CUDA function `name` in `path` (from its definition to the
    matching closing brace)."""
    text = open(path).read()
    i = text.find(f" {name}(")
    if i < 0:
        return None
    start = text.rfind("\n", 0, i) + 1
    j = text.find("{", i)
    depth = 0
    for k in range(j, len(text)):
        if text[k] == "{":
            depth += 1
        elif text[k] == "}":
            depth -= 1
            if depth == 0:
                return text[start:k + 1]
    return None


def traffic_for(kernel, units):
    """Per-launch DRAM bytes (read + write) of `kernel` from the committed ncu
    capture, scaled to `units` elements; None when the kernel's source text
    changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel)
    if not e:
        return None
    src = _function_source(os.path.join(ROOT, e["file"]), e["function"])
    if src is None or hashlib.sha256(src.encode()).hexdigest() != e["sha256"]:
        return None
    return int(e["bytes_per_unit"] * units)


def roofline_entry(dom, kern, n, A, st, peak, peak_src, total_ms, world):
    """The `roofline` object for the dominant kernel `dom`: algorithmic bytes
    per launch over its mean live launch time, against the measured copy
    bandwidth `peak` (GB/s).  `kern` maps kernel stage names to their live
    launch times (ms).  `traffic` is the committed per-launch DRAM traffic of
    that kernel (None when its source changed since the capture), and
    `traffic_frac` the DRAM bandwidth that traffic amounts to at the live
    launch time, as a fraction of the same peak."""
    if not dom:
        return None
    per_launch_ms = sum(kern[dom]) / len(kern[dom])
    byts = kernel_bytes(dom, n, A, st, 4)
    if not byts:
        return None
    achieved = byts / (per_launch_ms / 1e3) / 1e9
    traffic = traffic_for(dom, st["lr_n"] if dom.startswith("k_lr") else st["T"])
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_frac": (round(traffic / (per_launch_ms / 1e3) / 1e9 / peak, 4)
                             if traffic else None),
            "kernel": dom, "algorithmic_bytes": int(byts),
            "launch_ms": round(per_launch_ms, 4), "peak_source": peak_src,
            "share_of_step": round(sum(kern[dom]) / total_ms, 3) if world == 1 else None}


# ----------------------------------------------------------------- oracle (CPU baseline)

def oracle_edges_per_s(g, reps=1):
    import oracle
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
        oracle.euler_tour(g.n, tu, tv, g.root)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return g.m / t, t


# ----------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2603_11645_gb300 as rst
    from paper_2603_11645_gb300 import graphs, multi

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L = rst.lib()
    L.rst_launch_count.restype = ctypes.c_longlong
    L.rst_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.rst_profile_only.argtypes = [ctypes.c_char_p]
    L.rst_profile_only.restype = None
    L.rst_last_stats.argtypes = [ctypes.c_void_p, ctypes.c_int]

    g = graphs.workload_grid4096()
    from paper_2603_11645_gb300 import autotune
    tuning = autotune.apply(g.n, g.A)  # the tuned knobs of this size bucket (defaults if untuned)
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    par = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(strategy="cc_euler"):
        rst.build(off, col, g.root, strategy, out=par)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)

    def timed(nsteps, only=None):
        """nsteps steps, L2 flushed before each (outside the timed window),
        with the stage marks named in `only` recorded (None: every mark)."""
        L.rst_profile_only(only.encode() if only else None)
        L.rst_profile_enable(1)
        evs = []
        for _ in range(nsteps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        ms = (ctypes.c_float * 4096)()
        names = (ctypes.c_char_p * 4096)()
        k = L.rst_profile_read(ms, names, 4096)
        L.rst_profile_enable(0)
        L.rst_profile_only(None)
        seq = [(names[i].decode(), ms[i]) for i in range(k)]
        return [a.elapsed_time(b) for a, b in evs], seq

    # 1. the stage breakdown, on its own instrumented steps: an event between
    # every two stages (which also keeps each kernel from being scheduled while
    # the previous one drains, so these steps run a little slower)
    diag_steps = max(3, min(args.steps, 10))
    _, seq = timed(diag_steps)
    stages = {}
    for nm, v in seq:
        stages.setdefault(nm, []).append(v)
    kern = {nm: v for nm, v in stages.items() if nm.startswith("k_")}
    dom = max(kern, key=lambda nm: sum(kern[nm])) if kern else None
    pred = None  # the mark that opens the dominant kernel's stage
    for i, (nm, _) in enumerate(seq):
        if nm == dom and i > 0:
            pred = seq[i - 1][0]
            break
    stage_summary = {nm: round(sum(v) / diag_steps, 4) for nm, v in
                     sorted(stages.items(), key=lambda kv: -sum(kv[1]))}

    # 2. the timed region: K steps with only the two marks around the dominant
    # kernel recorded (its live launch time for the roofline)
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = L.rst_launch_count()
    step_ms, seq = timed(args.steps, f"{pred},{dom}" if dom and pred else None)
    launches = L.rst_launch_count() - launches0
    clk = clocks.stop()
    total_ms = multi.max_over_ranks(sum(step_ms), dev)  # the slowest replica
    value = multi.whole_job_rate(g.m * args.steps, world, total_ms / 1e3)
    if dom:
        live = [v for nm, v in seq if nm == dom]
        if live:
            kern = dict(kern, **{dom: live})
    stats = (ctypes.c_longlong * 8)()
    L.rst_last_stats(stats, 8)
    st = {"rounds": stats[0], "c1": stats[1], "E2": stats[2], "T": stats[3], "nroots": stats[4],
          "lr_levels": stats[5], "lr_n": stats[6]}
    peak, peak_src = measured_peaks()
    roofline = roofline_entry(dom, kern, g.n, g.A, st, peak, peak_src, total_ms, world)

    # end to end through the C ABI from pinned host buffers
    off_h = torch.from_numpy(g.offsets).pin_memory()
    col_h = torch.from_numpy(g.cols).pin_memory()
    par_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    off_d = torch.empty_like(off)
    col_d = torch.empty_like(col)
    e2e_steps = max(1, min(args.steps, 10))
    for _ in range(max(2, min(args.warmup, 3))):  # untimed: first copies from freshly pinned pages
        off_d.copy_(off_h, non_blocking=True)
        col_d.copy_(col_h, non_blocking=True)
        rst.build(off_d, col_d, g.root, "cc_euler", out=par)
        par_h.copy_(par, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = []
    for _ in range(e2e_steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        off_d.copy_(off_h, non_blocking=True)
        col_d.copy_(col_h, non_blocking=True)
        rst.build(off_d, col_d, g.root, "cc_euler", out=par)
        par_h.copy_(par, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = multi.max_over_ranks(sum(e2e_ms), dev)
    e2e_value = multi.whole_job_rate(g.m * e2e_steps, world, e2e_total / 1e3)
    e2e_streamed = run_e2e_streamed(rst, g, off, col, par, off_h, col_h, dev, stream, e2e_steps, world)

    # the library's own GPU BFS on the same graph (the step-bound baseline)
    bfs_ms = []
    step("bfs")
    for _ in range(args.bfs_steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step("bfs")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        bfs_ms.append(e0.elapsed_time(e1))
    L.rst_last_stats(stats, 8)
    bfs_levels = stats[5]
    bfs_med = statistics.median(bfs_ms)
    ms_step = total_ms / args.steps

    # the same search with the level loop on the device (no host round trip per
    # level): one launch per level inside a CUDA-graph while node, and one
    # persistent cooperative launch for all levels
    dev_bfs = {}
    for strat in ("bfs_device", "bfs_persistent"):
        c0 = L.rst_launch_count()
        step(strat)
        nl = L.rst_launch_count() - c0
        dev_bfs[strat] = (_time(lambda: step(strat), args.bfs_steps, torch, dev, stream, flush), nl)
    bfsd_med, bfsd_launches = dev_bfs["bfs_device"]
    bfsp_med, bfsp_launches = dev_bfs["bfs_persistent"]

    # PR-RST on the same graph
    pr_ms = []
    step("pr_rst")
    for _ in range(args.bfs_steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step("pr_rst")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pr_ms.append(e0.elapsed_time(e1))
    pr_med = statistics.median(pr_ms)

    # sampled union-find connectivity + the same Euler rooting (non-deterministic tree)
    fast_ms = _time(lambda: step("cc_fast"), max(3, args.bfs_steps), torch, dev, stream, flush)

    # blocks and cut vertices on top of the Euler tour (Tarjan-Vishkin)
    bcc_ms = _time(lambda: rst.bcc(off, col), max(3, args.bfs_steps), torch, dev, stream, flush)
    _, bcc_cut, bcc_blocks = rst.bcc(off, col)
    bcc_rep = {"value": g.m / (bcc_ms / 1e3), "unit": "edges/s", "ms_per_step": bcc_ms,
               "blocks": bcc_blocks, "cut_vertices": int(bcc_cut.sum().item())}

    # edge insertions: the forest of the graph with 45% of its edges held back,
    # then those edges inserted with PR-RST graft and reversal
    ins_rep = run_insert(g, dev, stream, rst, graphs, torch, max(3, args.bfs_steps), total_ms / args.steps)

    # tree shape (Fig. 2): heights of the trees each strategy returns
    heights = {}
    for strat in ("cc_euler", "bfs", "pr_rst", "cc_fast"):
        step(strat)
        heights[strat] = rst.tree_depth(par, want_depths=False)[1]

    cpu_on = world == 1 and not args.no_cpu_baseline
    grid256 = run_grid256(args, dev, stream, rst, graphs, torch, cpu_on)
    batch = None if args.no_batch else run_batch(args, dev, stream, rst, graphs, torch, rank, world, cpu_on)
    families = None if args.no_families else run_families(args, dev, stream, rst, graphs, torch, peak, cpu_on)
    selector = run_selector_report(off, col, g.root, torch)

    out = None
    if rank == 0:
        cpu = None
        if cpu_on:
            v, t = oracle_edges_per_s(g, 1)
            cpu = {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                   "sample": f"one run of the sequential oracle (Kruskal over (min,max) keys + "
                             f"sequential Euler tour) on the full 4096x4096 workload, {t:.1f} s",
                   **host_cpu()}
        out = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "strategy": "cc_euler",
                       "l2": "L2 flushed (258 MB write) before every timed step; inputs also exceed L2",
                       "parallelism": "replicas" if world > 1 else "single GPU", "tuning": tuning},
            "e2e": {"value": e2e_value, "unit": "edges/s",
                    "h2d_bytes_per_step": int(g.offsets.nbytes + g.cols.nbytes),
                    "d2h_bytes_per_step": int(4 * g.n),
                    "schedule": "serial: each step copies its CSR in, builds, copies the parents out"},
            "e2e_streamed": e2e_streamed,
            "gpu_launches": int(launches),
            "roofline": roofline,
            "roofline_step": step_roofline(g.n, g.A, st["T"], 4, ms_step, peak),
            "cpu_baseline": cpu,
            "clocks": clk,
            "bfs": {"value": g.m / (bfs_med / 1e3), "unit": "edges/s", "ms_per_step": bfs_med,
                    "levels": int(bfs_levels), "loop": "host reads the frontier size every level",
                    "cc_euler_speedup": bfs_med / ms_step},
            "bfs_device": {"value": g.m / (bfsd_med / 1e3), "unit": "edges/s", "ms_per_step": bfsd_med,
                           "levels": int(bfs_levels), "launches": int(bfsd_launches),
                           "loop": "one kernel per level inside a CUDA-graph while loop",
                           "cc_euler_speedup": bfsd_med / ms_step},
            "bfs_persistent": {"value": g.m / (bfsp_med / 1e3), "unit": "edges/s", "ms_per_step": bfsp_med,
                               "levels": int(bfs_levels), "launches": int(bfsp_launches),
                               "loop": "all levels in one cooperative launch, a grid barrier per level",
                               "cc_euler_speedup": bfsp_med / ms_step},
            "pr_rst": {"value": g.m / (pr_med / 1e3), "unit": "edges/s", "ms_per_step": pr_med,
                       "cc_euler_speedup": pr_med / ms_step},
            "cc_fast": {"value": g.m / (fast_ms / 1e3), "unit": "edges/s", "ms_per_step": fast_ms,
                        "note": "sampled union-find CC + the same Euler rooting; valid RST, tree not unique"},
            "tree_height": heights,
            "bcc": bcc_rep,
            "insert": ins_rep,
            "grid256": grid256,
            "batch": batch,
            "families": families,
            "selector": selector,
            "stats": st,
            "stage_ms": stage_summary,
            "stage_ms_note": "mean per step over a separate pass of instrumented steps (an event between every "
                             "two stages); the timed steps record only the two events around the roofline kernel",
        }
    return out


def run_batch(args, dev, stream, rst, graphs, torch, rank=0, world=1, cpu_on=False):
    """4096 mixed graphs: one rst_build_batch call vs one rst_build call per
    graph.  With several ranks the graphs are split by arc count (LPT) and
    each rank builds its share; times are the slowest rank's."""
    from paper_2603_11645_gb300 import multi
    full = graphs.workload_batch(hi=args.batch_hi)
    b = full
    if world > 1:
        shard = multi.lpt_shards([g.A for g in full.graphs], world)[rank]
        b = graphs.pack_batch([full.graphs[i] for i in shard])
    from paper_2603_11645_gb300 import autotune
    autotune.apply(b.N, b.A)
    off = torch.from_numpy(b.offsets).to(dev)
    col = torch.from_numpy(b.cols).to(dev)
    vo = torch.from_numpy(b.vtx_off).to(dev)
    ao = torch.from_numpy(b.arc_off).to(dev)
    roots = torch.from_numpy(b.roots).to(dev)
    par = torch.empty(b.N, dtype=torch.int32, device=dev)
    for _ in range(2):
        rst.build_batch(off, col, vo, ao, roots, out=par)
    times = []
    for _ in range(max(3, min(args.steps, 10))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rst.build_batch(off, col, vo, ao, roots, out=par)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    batched = multi.max_over_ranks(statistics.median(times), dev)
    # per-graph launches over the same resident data (zero-copy views)
    views = []
    for g_i, g in enumerate(b.graphs):
        o0 = int(b.vtx_off[g_i]) + g_i
        a0, a1 = int(b.arc_off[g_i]), int(b.arc_off[g_i + 1])
        views.append((off[o0:o0 + g.n + 1], col[a0:a1], g.root, par[int(b.vtx_off[g_i]):int(b.vtx_off[g_i + 1])]))
    for o, c, r, p in views[:64]:
        rst.build(o, c, r, out=p)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for o, c, r, p in views:
        rst.build(o, c, r, out=p)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    per_graph = multi.max_over_ranks(e0.elapsed_time(e1), dev)
    cpu = None
    if cpu_on and rank == 0:
        import oracle
        t0 = time.perf_counter()
        for gr in full.graphs:
            lab, tu, tv = oracle.cc_kruskal(gr.n, gr.offsets, gr.cols)
            oracle.euler_tour(gr.n, tu, tv, gr.root)
        t = time.perf_counter() - t0
        cpu = {"value": full.m / t, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"one pass of the sequential oracle (Kruskal + Euler tour) over all "
                         f"{full.G} graphs of the batch, {t:.1f} s", **host_cpu()}
    return {"ranks": world, "cpu_baseline": cpu,
            "workload": f"{full.G} graphs (grid / chain+chords / R-MAT in turn), n log-uniform "
                        f"1K-{args.batch_hi // 1024}K, "
                        f"{full.N} vertices, {full.A} arcs, int32 packed CSR"
                        + (f", split over {world} ranks by arc count" if world > 1 else ""),
            "graphs": full.G, "m": full.m, "batched_ms": batched, "per_graph_ms": per_graph,
            "batched_value": full.m / (batched / 1e3), "per_graph_value": full.m / (per_graph / 1e3),
            "unit": "edges/s", "speedup": per_graph / batched}


def run_insert(g, dev, stream, rst, graphs, torch, reps, rebuild_ms):
    """Edge insertions (rst_insert_edges with the canonical flag: the forests
    come from rst_build).  Two forests of the headline grid: 45% of its edges
    held back (55% kept, above the square lattice's bond-percolation
    threshold of 50%: one giant, deep tree beside ~1M small ones) and 60% held
    back (40% kept, below it: small trees only).  Batches of the held-back
    edges in a seeded order (1,000, 100,000, and for the first forest all of
    them), each beside a full CC+Euler rebuild of the graph."""
    import numpy as np
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    col = g.cols.astype(np.int64)
    fwd = src < col
    lo, hi = src[fwd], col[fwd]
    h = (lo * 0x9E3779B1 + hi * 0x85EBCA77 + 11) % 1000003
    out = {"note": "PR-RST rounds from the existing forest over the inserted edges only; batches of at most "
                   "n/64 edges run them sparsely (walks to roots, per-tree path reversal) while every walk "
                   "stays within insert_walk_limit steps, and the canonical flag re-roots only merged trees"}
    for name, thr, sizes in (("held_back_45pct", 450000, (1000, 100000, None)),
                             ("held_back_60pct", 600000, (1000, 100000))):
        drop = h < thr
        g0 = graphs.from_edges(g.n, lo[~drop], hi[~drop], root=g.root)
        held = np.stack([lo[drop], hi[drop]], 1).astype(np.int32)
        held = held[np.random.default_rng(12).permutation(len(held))]
        off0 = torch.from_numpy(g0.offsets).to(dev)
        col0 = torch.from_numpy(g0.cols).to(dev)
        base = rst.build(off0, col0, g.root, "cc_euler")
        _, height = rst.tree_depth(base, want_depths=False)
        work = torch.empty_like(base)
        batches = {}
        for k in sizes:
            k = len(held) if k is None else k
            uv = torch.from_numpy(np.ascontiguousarray(held[:k])).to(dev)
            ts = []
            for i in range(reps + 1):
                work.copy_(base)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rst.insert_edges(work, uv, g.root, canonical=True)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if i:
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            batches[str(k)] = {"ms": ms, "rebuild_ms": rebuild_ms, "speedup_over_rebuild": rebuild_ms / ms}
        out[name] = {"workload": f"4096x4096 grid forest with {int(drop.sum())} edges held back, then batches "
                                 f"of them inserted", "trees_before":
                         int((base.cpu() == torch.arange(g.n, dtype=torch.int32)).sum()),
                     "height_before": int(height), "batches": batches}
        del off0, col0, base, work
    return out


def _time(fn, reps, torch, dev, stream, flush=None):
    fn()
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _stats(L):
    stats = (ctypes.c_longlong * 8)()
    L.rst_last_stats(stats, 8)
    return {"rounds": stats[0], "c1": stats[1], "E2": stats[2], "T": stats[3], "nroots": stats[4],
            "lr_levels": stats[5], "lr_n": stats[6]}


def run_families(args, dev, stream, rst, graphs, torch, peak, cpu_on):
    """The power-law workload: R-MAT scale 24, edge factor 16, (0.57, 0.19,
    0.19, 0.05), symmetrised, deduplicated, connected to vertex 0, int64
    offsets, root 0.  Every strategy, the whole CC+Euler step against the
    byte model, and the sequential oracle on the same graph."""
    g = graphs.workload_rmat24()
    from paper_2603_11645_gb300 import autotune
    autotune.apply(g.n, g.A)
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    par = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    out = {"workload": f"R-MAT scale 24, edge factor 16, (0.57,0.19,0.19,0.05), symmetrised, "
                       f"deduplicated, connected to 0, int64 offsets, root 0: {g.n} vertices, "
                       f"{g.m} edges ({g.A} arcs)", "n": g.n, "m": g.m}
    L = rst.lib()
    for strat in ("cc_euler", "bfs", "bfs_device", "bfs_persistent", "pr_rst", "cc_fast"):
        if strat not in rst.STRATEGIES:
            continue
        reps = max(3, min(args.steps, 10)) if strat == "cc_euler" else 3
        ms = _time(lambda: rst.build(off, col, g.root, strat, out=par), reps, torch, dev, stream, flush)
        out[strat] = {"ms": ms, "value": g.m / (ms / 1e3), "unit": "edges/s"}
        if strat == "cc_euler":
            st = _stats(L)
            out["cc_euler"]["roofline_step"] = step_roofline(g.n, g.A, st["T"], 8, ms, peak)
            out["cc_euler"]["stats"] = st
    out["cc_euler_speedup_over_bfs"] = out["bfs"]["ms"] / out["cc_euler"]["ms"]
    ms = _time(lambda: rst.bcc(off, col), 3, torch, dev, stream, flush)
    _, cut, nb = rst.bcc(off, col)
    out["bcc"] = {"ms": ms, "value": g.m / (ms / 1e3), "unit": "edges/s", "blocks": nb,
                  "cut_vertices": int(cut.sum().item())}
    if cpu_on:
        v, t = oracle_edges_per_s(g, 1)
        out["cpu_baseline"] = {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": f"one run of the sequential oracle (Kruskal + Euler tour) on "
                                         f"the full R-MAT scale-24 graph, {t:.1f} s", **host_cpu()}
    del off, col, par, flush
    torch.cuda.empty_cache()
    return {"rmat24": out}


def run_grid256(args, dev, stream, rst, graphs, torch, cpu_on):
    """The 256 x 256 permuted grid (65,536 vertices, root = the permuted
    corner): small enough to live in L2, so it measures latency and launch
    counts rather than bandwidth."""
    g = graphs.workload_grid256()
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    par = torch.empty(g.n, dtype=torch.int32, device=dev)
    L = rst.lib()
    out = {"workload": "grid 256x256 4-neighbour, ids permuted by seed 1, root = permuted corner, "
                       "int32 CSR (65,536 vertices, 130,560 edges)", "n": g.n, "m": g.m}
    for strat in ("cc_euler", "bfs", "bfs_device", "bfs_persistent", "pr_rst"):
        if strat not in rst.STRATEGIES:
            continue
        rst.build(off, col, g.root, strat, out=par)
        c0 = L.rst_launch_count()
        rst.build(off, col, g.root, strat, out=par)
        launches = L.rst_launch_count() - c0
        ms = _time(lambda: rst.build(off, col, g.root, strat, out=par), 20, torch, dev, stream)
        out[strat] = {"us": round(ms * 1e3, 1), "value": g.m / (ms / 1e3), "unit": "edges/s",
                      "launches": int(launches)}
    if cpu_on:
        import oracle
        ts = []
        for _ in range(6):
            t0 = time.perf_counter()
            lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
            oracle.euler_tour(g.n, tu, tv, g.root)
            ts.append(time.perf_counter() - t0)
        t = statistics.median(ts[1:])
        out["cpu_baseline"] = {"value": g.m / t, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": "sequential oracle (Kruskal + Euler tour) on the full graph, "
                                         "median of 5 runs after 1 warm-up", **host_cpu()}
    return out


def run_selector_report(off, col, root, torch, count=24):
    """The learned selector measured in this run: the first `count` held-out
    graphs of the selector workload (seeds 9000+i, the four families in turn,
    n log-uniform in [2^16, 2^22]) are generated, all three strategies are
    timed on each (BFS capped as in training), and rst_select's choice (GPU
    features, GPU network) is scored: regret = mean (t_chosen - t_best) /
    t_best, beside always choosing CC+Euler.  Also the cost of one rst_select
    call on the headline graph and the stored 200-graph report."""
    from paper_2603_11645_gb300 import selector as S
    model = S.load_default()
    if model is None:
        return None
    t0 = time.perf_counter()
    for _ in range(5):
        choice, pred = S.select(off, col, root)
    sel_ms = (time.perf_counter() - t0) / 5 * 1e3
    rows = []
    for g in S.family_graphs("heldout", range(count)):  # the pool is idle while a chunk is timed
        o = torch.from_numpy(g.offsets).cuda()
        c = torch.from_numpy(g.cols).cuda()
        ts, cens = S.time_strategies(o, c, g.root)
        ch, _ = S.select(o, c, g.root)
        rows.append((g.meta.get("family", "?"), g.n, ts, S.STRATS.index(ch), cens))
        del o, c
    T = [r[2] for r in rows]
    best = [min(range(3), key=lambda k: t[k]) for t in T]

    def reg(ch):
        return sum((t[k] - t[b]) / t[b] for t, k, b in zip(T, ch, best)) / len(T)

    chosen = [r[3] for r in rows]
    rep = model.get("heldout_report", {})
    return {"heldout_regret": reg(chosen), "always_cc_euler_regret": reg([1] * len(T)),
            "always_bfs_regret": reg([0] * len(T)),
            "heldout_graphs": len(T), "margin": model.get("margin"),
            "choice_counts": {s: chosen.count(k) for k, s in enumerate(S.STRATS)},
            "best_counts": {s: best.count(k) for k, s in enumerate(S.STRATS)},
            "bfs_censored": sum(r[4] for r in rows),
            "workload": f"held-out graphs 0..{count - 1} of the selector workload (grid / chain+chords / "
                        f"R-MAT / random 4-regular in turn, n log-uniform 2^16..2^22), timed live; choices by "
                        f"rst_select (features and network on the GPU)",
            "choice_on_headline": choice, "select_ms": sel_ms,
            "stored_report": {k: rep.get(k) for k in ("heldout_graphs", "selector_regret",
                                                      "always_cc_euler_regret", "selector_choice_counts",
                                                      "oracle_choice_counts")}}


PROFILE_STRATEGIES = ("cc_euler", "bfs", "bfs_device", "bfs_persistent", "pr_rst", "cc_fast", "bcc", "verify",
                      "depth", "euler_root", "select", "mlp", "insert")


def run_profile_case(args):
    """One path alone, W warm-up + K calls and no timing, on a SIDE x SIDE
    permuted grid (seed 2): the command the ncu captures run.  The strategy
    is --profile-strategy (default cc_euler); "euler_root" roots the grid's
    spanning forest from its edge list (radix sort + tour), "select" runs the
    selector's features and network, "mlp" the training kernels on a batch of
    SIDE feature rows, "insert" inserts 1,000 edges into the forest of the
    grid with 45% of its edges held back."""
    import numpy as np
    import torch

    import paper_2603_11645_gb300 as rst
    from paper_2603_11645_gb300 import graphs
    side = args.profile_case
    strat = args.profile_strategy
    calls = args.warmup + args.steps
    if args.profile_graph == "rmat":  # R-MAT of about SIDE^2 vertices, connected, int64 offsets
        import math
        g = graphs.rmat(int(round(math.log2(side * side))), 16, seed=3, connect=True, offsets_bits=64)
    else:
        g = graphs.grid(side, side, seed=2, permute=True, root="random")
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    if strat in ("cc_euler", "bfs", "bfs_device", "bfs_persistent", "pr_rst", "cc_fast"):
        for _ in range(calls):
            rst.build(off, col, g.root, strat, out=par)
    elif strat == "bcc":
        for _ in range(calls):
            rst.bcc(off, col)
    elif strat == "verify":
        rst.build(off, col, g.root, "cc_euler", out=par)
        for _ in range(calls):
            rst.verify(off, col, g.root, par)
    elif strat == "depth":
        rst.build(off, col, g.root, "cc_euler", out=par)
        for _ in range(calls):
            rst.tree_depth(par)
    elif strat == "euler_root":
        labels, uv, T = rst.cc(off, col)
        uv = uv.clone()
        for _ in range(calls):
            rst.euler_root(g.n, uv, g.root, with_rank=True)
    elif strat == "select":
        from paper_2603_11645_gb300 import selector as S
        S.load_default()
        for _ in range(calls):
            S.select(off, col, g.root)
    elif strat == "mlp":
        from paper_2603_11645_gb300 import selector as S
        rng = np.random.default_rng(3)
        X = rng.normal(size=(side, S.F))
        Tt = np.exp(rng.normal(size=(side, S.O)))
        for _ in range(calls):
            S.train(X, Tt, epochs=5, lr=1e-3, seed=1)
    elif strat == "insert":
        src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
        c64 = g.cols.astype(np.int64)
        fwd = src < c64
        lo, hi = src[fwd], c64[fwd]
        drop = ((lo * 0x9E3779B1 + hi * 0x85EBCA77 + 11) % 1000003) < 450000
        g0 = graphs.from_edges(g.n, lo[~drop], hi[~drop], root=g.root)
        uv = torch.from_numpy(np.stack([lo[drop], hi[drop]], 1)[:1000].astype(np.int32)).cuda()
        base = rst.build(torch.from_numpy(g0.offsets).cuda(), torch.from_numpy(g0.cols).cuda(), g.root)
        work = torch.empty_like(base)
        for _ in range(calls):
            work.copy_(base)
            rst.insert_edges(work, uv, g.root)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": g.name, "strategy": strat, "n": g.n, "A": g.A, "calls": calls}))


# ----------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2603_11645_gb300 import graphs
    import oracle
    # bounded sample of the workload: the same family at 2048 x 2048 (seed 2)
    g = graphs.grid(2048, 2048, seed=2, permute=True, root="random")
    for _ in range(args.warmup):
        oracle_edges_per_s(g, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
        oracle.euler_tour(g.n, tu, tv, g.root)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = g.m * args.steps / total
    sample = ("sequential CPU oracle (Kruskal + Euler tour) per step on a 2048x2048 grid of the "
              "same family (4,194,304 vertices, 8,384,512 edges)")
    return {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "strategy": "cc_euler (oracle)"},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def launch_command(argv, gpus, port):
    """The torchrun command that starts `gpus` ranks of this script on one node
    (rendezvous on 127.0.0.1), used when --gpus N > 1 is given without a
    launcher."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *argv]


def _free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--bfs-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-families", action="store_true")
    ap.add_argument("--batch-hi", type=int, default=4096,
                    help="largest vertex count of the batch's graphs (262144: the literal 1K-256K size law)")
    ap.add_argument("--profile-case", type=int, default=0, metavar="SIDE",
                    help="only run one path (W warm-up + K calls, no timing) on a SIDE x SIDE grid of the "
                         "headline family; the command the ncu captures use")
    ap.add_argument("--profile-strategy", default="cc_euler", choices=PROFILE_STRATEGIES,
                    help="the path --profile-case runs")
    ap.add_argument("--profile-graph", default="grid", choices=["grid", "rmat"],
                    help="the graph --profile-case runs on: the permuted SIDE x SIDE grid, or R-MAT of "
                         "scale round(log2 SIDE^2) connected to vertex 0")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks and hand back their exit status
        sys.exit(subprocess.call(launch_command(sys.argv[1:], args.gpus, _free_port())))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but the launcher started {world} ranks")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
