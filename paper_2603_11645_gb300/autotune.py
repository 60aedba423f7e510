"""Offline tuning of the speed-only launch parameters, cached per size bucket.

The knobs (include/rst.h, rst_set_option) change how the work is split into
launches and samples, never a result:

* ``lr_spacing``: list-ranking splitter spacing K of the first level (one
  splitter per K tour arcs; sample rate 1/K; the deeper levels use 8);
* ``round_blocks_per_sm``: grid of the contraction-round kernels (the hook
  and resolve kernels cap it at the blocks their registers let reside);
* ``bfs_bottom_up_divisor``: BFS steps bottom-up while the frontier holds more
  than n / divisor vertices;
* ``bfs_device_blocks_per_sm`` / ``bfs_persistent_blocks_per_sm``: the grid of
  the device-driven BFS variants (a small grid keeps the per-level cost of
  deep, narrow searches low; a large one feeds the wide bottom-up levels);
* ``euler_block``: the block size (128/256/512) of the tour's grid-stride
  kernels;
* ``pr_levels_per_launch``: PR-RST's pointer-jumping levels per launch and
  host check (1..3), the counterpart of Section III-C's several pointer jumps
  per global synchronisation.

They stand where Section III-C fixes its own launch granularity empirically
(five pointer jumps per global synchronisation for PR-RST).  ``tune`` times
every value of one knob with the others held, keeps the fastest, and moves to
the next knob (coordinate descent), on one synthetic graph per bucket: a
permuted square grid for sparse buckets (mean degree <= 8) and an R-MAT graph
for dense ones.  ``apply`` looks up the bucket of a graph and sets its knobs.

    python -m paper_2603_11645_gb300.autotune --out paper_2603_11645_gb300/tuning.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics

KNOBS = {
    "round_blocks_per_sm": [2, 4, 8, 16],
    "lr_spacing": [16, 32, 64, 128, 256, 512],
    "bfs_bottom_up_divisor": [5, 10, 20, 40, 80],
    "bfs_device_blocks_per_sm": [1, 2, 4, 8],
    "bfs_persistent_blocks_per_sm": [1, 2, 4],
    "euler_block": [128, 256, 512],
    "pr_levels_per_launch": [1, 2, 3],
}
DEFAULTS = {"round_blocks_per_sm": 8, "lr_spacing": 16, "bfs_bottom_up_divisor": 20,
            "bfs_device_blocks_per_sm": 2, "bfs_persistent_blocks_per_sm": 1, "euler_block": 256,
            "pr_levels_per_launch": 1}
# the strategy whose time decides each knob
KNOB_STRATEGY = {"round_blocks_per_sm": "cc_euler", "lr_spacing": "cc_euler", "bfs_bottom_up_divisor": "bfs",
                 "bfs_device_blocks_per_sm": "bfs_device", "bfs_persistent_blocks_per_sm": "bfs_persistent",
                 "euler_block": "cc_euler", "pr_levels_per_launch": "pr_rst"}

# size buckets by log2 n (half-open), with the log2 n of the graph tuned on
BUCKETS = [(0, 14, 12), (14, 18, 16), (18, 22, 20), (22, 31, 24)]
DENSE_MAX_LOG2N = 22  # dense buckets are tuned on R-MAT up to this scale
TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def degree_class(n: int, m_arcs: int) -> str:
    """'sparse' for mean degree (arcs per vertex) <= 8, else 'dense'."""
    return "sparse" if n == 0 or m_arcs <= 8 * n else "dense"


def bucket_of(n: int, m_arcs: int, table: dict) -> dict | None:
    """The table entry whose log2 n range holds n and whose degree class is
    that of the graph (None if the table has no such entry)."""
    lg = math.log2(n) if n > 0 else 0.0
    cls = degree_class(n, m_arcs)
    for e in table.get("buckets", []):
        lo, hi = e["log2n"]
        if lo <= lg < hi and e["degree"] == cls:
            return e
    return None


def load(path: str = TUNING_PATH) -> dict | None:
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


def apply(n: int, m_arcs: int, table: dict | None = None) -> dict:
    """Set the knobs of the graph's bucket (defaults where the table has none)
    and return the options in force."""
    import paper_2603_11645_gb300 as rst
    table = table if table is not None else (load() or {})
    e = bucket_of(n, m_arcs, table)
    opts = dict(DEFAULTS)
    if e:
        opts.update({k: v for k, v in e["options"].items() if k in KNOBS})
    for k, v in opts.items():
        rst.set_option(k, v)
    return opts


def reset() -> None:
    import paper_2603_11645_gb300 as rst
    for k, v in DEFAULTS.items():
        rst.set_option(k, v)


def _graph_for(lg: int, cls: str, seed: int):
    from . import graphs
    if cls == "sparse":
        side = 1 << (lg // 2)
        return graphs.grid(side, (1 << lg) // side, seed=seed, permute=True, root="random")
    return graphs.rmat(min(lg, DENSE_MAX_LOG2N), 16, seed=seed, connect=True,
                       offsets_bits=64 if lg >= 22 else 32)


def _time_ms(fn, reps, torch):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_graph(g, reps: int = 5, knobs: dict | None = None) -> dict:
    """Coordinate descent over the knobs on one graph; returns the chosen
    options and the times seen (ms).  Leaves the defaults in force."""
    import torch

    import paper_2603_11645_gb300 as rst
    knobs = knobs or KNOBS
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    cur = dict(DEFAULTS)
    times = {}
    base = {}
    try:
        for s in set(KNOB_STRATEGY[k] for k in knobs):
            for k, v in cur.items():
                rst.set_option(k, v)
            base[s] = _time_ms(lambda: rst.build(off, col, g.root, s, out=par), reps, torch)
        for knob, values in knobs.items():
            s = KNOB_STRATEGY[knob]
            seen = {}
            for v in values:
                for k, x in cur.items():
                    rst.set_option(k, x)
                rst.set_option(knob, v)
                seen[v] = _time_ms(lambda: rst.build(off, col, g.root, s, out=par), reps, torch)
            best = min(seen, key=seen.get)
            cur[knob] = best
            times[knob] = {str(v): round(t, 4) for v, t in seen.items()}
        tuned = {}
        for s in base:
            for k, v in cur.items():
                rst.set_option(k, v)
            tuned[s] = _time_ms(lambda: rst.build(off, col, g.root, s, out=par), reps, torch)
    finally:
        reset()
    return {"options": cur, "times_ms": times,
            "default_ms": {s: round(t, 4) for s, t in base.items()},
            "tuned_ms": {s: round(t, 4) for s, t in tuned.items()}}


def tune(buckets=BUCKETS, classes=("sparse", "dense"), reps: int = 5, seed: int = 7) -> dict:
    import torch
    table = {"device": torch.cuda.get_device_name(0), "reps": reps, "seed": seed,
             "knobs": KNOBS, "defaults": DEFAULTS, "buckets": []}
    for lo, hi, lg in buckets:
        for cls in classes:
            g = _graph_for(lg, cls, seed)
            r = tune_graph(g, reps)
            table["buckets"].append({"log2n": [lo, hi], "degree": cls,
                                     "graph": f"{g.name}: n={g.n}, arcs={g.A}", **r})
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TUNING_PATH)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    table = tune(reps=args.reps)
    with open(args.out, "w") as fh:
        json.dump(table, fh, indent=1)
    for e in table["buckets"]:
        print(e["log2n"], e["degree"], e["options"], e["default_ms"], e["tuned_ms"])


if __name__ == "__main__":
    main()
