"""Learned strategy selector: data generation, GPU training, GPU inference.

The library's own timings of BFS, CC+Euler and PR-RST on seeded graphs train a
12-64-64-3 network (rst_mlp_train: forward, backward and Adam kernels on the
GPU) that predicts each strategy's log-time from 12 cheap features
(rst_selector_features, computed on the GPU).  rst_select / rst_build(RST_AUTO)
run the features, the network and the choice on the GPU: the smallest
prediction wins, and CC+Euler is kept when another strategy's predicted gain
is below a margin.  This module only moves data to and from those calls.

Graph families (seeded; training seeds 5000+i, held-out seeds 9000+i), in
turn: grids with aspect ratio log-uniform in [1, 4096], paths with uniformly
random chords at density log-uniform in [1e-6, 1e-1], R-MAT graphs of scale
round(log2 n) in [16, 22] connected to vertex 0, and random 4-regular graphs;
vertex counts log-uniform in [2^16, 2^22].  BFS runs are capped at
BFS_LEVEL_CAP levels; a capped run is labelled with the time spent up to the
cap (a lower bound far above the best strategy's time, so it is never the
argmin and regret stays exact).
"""
from __future__ import annotations

import ctypes
import csv
import json
import math
import os
import time

import numpy as np

from . import graphs

F, H, O = 12, 64, 3
NPARAM = H * F + H + H * H + H + O * H + O
STRATS = ("bfs", "cc_euler", "pr_rst")
CHOICE_INDEX = {1: 0, 2: 1, 3: 2}  # rst_strategy code -> position in STRATS
BFS_LEVEL_CAP = 1024
LOG2N_RANGE = (16, 22)
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")
FEATURE_NAMES = ["log2_n", "log2_m", "mean_deg", "deg_cv", "deg_skew", "log2_maxdeg", "frac_deg_le2",
                 "log2_probe_reached", "log2_probe_growth", "log2_ecc_est", "log2_r1_comp_frac",
                 "surviving_edge_frac"]


def _lib():
    from . import lib
    L = lib()
    P, I, I32, I64, Fl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    L.rst_selector_features.argtypes = [P, I, P, I64, I64, I32, P, P]
    L.rst_selector_load.argtypes = [P, P, Fl]
    L.rst_select.argtypes = [P, I, P, I64, I64, I32, P, P, P]
    L.rst_selector_predict.argtypes = [P, I, P, P, P]
    L.rst_mlp_forward.argtypes = [P, P, I, P, P]
    L.rst_mlp_loss_grad.argtypes = [P, P, P, I, P, P, P]
    L.rst_mlp_adam.argtypes = [P, P, P, P, I, I, Fl, Fl, Fl, Fl, P]
    L.rst_mlp_train.argtypes = [P, P, P, I, I, Fl, P, P, P, P]
    L.rst_set_option.argtypes = [ctypes.c_char_p, ctypes.c_longlong]
    for fn in ("rst_selector_features", "rst_selector_load", "rst_select", "rst_selector_predict", "rst_mlp_forward",
               "rst_mlp_loss_grad", "rst_mlp_adam", "rst_mlp_train", "rst_set_option"):
        getattr(L, fn).restype = I
    return L


def _check(fn, code):
    if code != 0:
        from . import RstError
        raise RstError(fn, code)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ graph families

def family_graph(i: int, split: str = "train") -> graphs.Graph:
    seed = (5000 if split == "train" else 9000) + i
    r = graphs.uniform(4, 1 << 30, seed * 7919 + 11).astype(np.float64) / (1 << 30)
    fam = i % 4
    lo, hi = LOG2N_RANGE
    n = int(round(math.exp(math.log(2 ** lo) + r[0] * (math.log(2 ** hi) - math.log(2 ** lo)))))
    if fam == 0:
        aspect = math.exp(r[1] * math.log(4096.0))
        Hh = max(1, int(round(math.sqrt(n / aspect))))
        W = max(1, n // Hh)
        g = graphs.grid(W, Hh, seed=seed, permute=True, root="random")
    elif fam == 1:
        d = math.exp(math.log(1e-6) + r[1] * (math.log(1e-1) - math.log(1e-6)))
        g = graphs.chain_chords(n, d, seed=seed)
        g.root = int(graphs.uniform(1, n, seed + 3)[0])
    elif fam == 2:
        scale = max(lo, min(hi, int(round(math.log2(n)))))
        g = graphs.rmat(scale, 16, seed=seed, connect=True, offsets_bits=32)
    else:
        g = graphs.random_4regular(max(n, 5), seed=seed)
    g.meta["split"] = split
    g.meta["index"] = i
    return g


def _family_graph_args(args):
    return family_graph(*args)


def _worker_init(threads: int):
    os.environ["GG_THREADS"] = str(threads)  # the generator's own threads per worker


def family_graphs(split: str, indices, workers: int | None = None):
    """The split's graphs in index order.  They are generated a chunk at a time
    by a pool of spawned worker processes (no CUDA in them); the pool is idle
    while the caller consumes a chunk, so timings taken meanwhile see no
    competing host load (the host-stepped strategies are sensitive to it)."""
    import multiprocessing as mp
    indices = list(indices)
    cores = os.cpu_count() or 2
    workers = workers or max(1, min(8, cores // 2))
    if workers <= 1 or len(indices) <= 1:
        for i in indices:
            yield family_graph(i, split)
        return
    ctx = mp.get_context("spawn")
    chunk = 4 * workers
    with ctx.Pool(workers, initializer=_worker_init, initargs=(max(1, cores // workers),)) as pool:
        for c0 in range(0, len(indices), chunk):
            part = [(i, split) for i in indices[c0:c0 + chunk]]
            for g in pool.map(_family_graph_args, part, chunksize=1):
                yield g


# ------------------------------------------------------------------ GPU calls

def features(off, col, root: int) -> np.ndarray:
    import torch
    L = _lib()
    f = np.zeros(F, dtype=np.float32)
    bits = 64 if off.dtype == torch.int64 else 32
    code = L.rst_selector_features(ctypes.c_void_p(off.data_ptr()), bits, ctypes.c_void_p(col.data_ptr()),
                                   off.numel() - 1, col.numel(), int(root), f.ctypes.data, _stream())
    _check("rst_selector_features", code)
    return f


def time_strategies(off, col, root: int, reps: int = 3):
    """Median wall time (s, CUDA events) of each strategy; BFS capped."""
    import torch
    from . import build, RstError
    L = _lib()
    out = torch.empty(off.numel() - 1, dtype=torch.int32, device=off.device)
    times, censored = [], False
    for strat in STRATS:
        if strat == "bfs":
            L.rst_set_option(b"bfs_max_levels", BFS_LEVEL_CAP)
        ts = []
        for k in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            try:
                build(off, col, root, strat, out=out)
            except RstError as e:
                if strat != "bfs" or e.code != 4:
                    raise
                censored = True
            e1.record()
            torch.cuda.synchronize()
            if k > 0:
                ts.append(e0.elapsed_time(e1) / 1e3)
        if strat == "bfs":
            L.rst_set_option(b"bfs_max_levels", 0)
        times.append(float(np.median(ts)))
    return times, censored


def generate_dataset(split: str, count: int, path: str, reps: int = 3, log_every: int = 100):
    """Features and timings of `count` graphs of the split, written as CSV."""
    import torch
    rows = []
    t0 = time.time()
    for i, g in enumerate(family_graphs(split, range(count))):
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        f = features(off, col, g.root)
        ts, cens = time_strategies(off, col, g.root, reps)
        rows.append([split, i, g.meta.get("family", "?"), g.n, g.m] + [float(x) for x in f] + ts + [int(cens)])
        del off, col
        if log_every and (i + 1) % log_every == 0:
            print(f"[{split}] {i + 1}/{count} graphs, {time.time() - t0:.0f} s", flush=True)
    header = ["split", "index", "family", "n", "m"] + FEATURE_NAMES + [f"t_{s}" for s in STRATS] + ["bfs_censored"]
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(header)
        w.writerows(rows)
    return path


def load_dataset(path: str):
    with open(path) as fh:
        r = csv.DictReader(fh)
        rows = list(r)
    X = np.array([[float(row[k]) for k in FEATURE_NAMES] for row in rows], dtype=np.float64)
    Tt = np.array([[float(row[f"t_{s}"]) for s in STRATS] for row in rows], dtype=np.float64)
    fam = [row["family"] for row in rows]
    return X, Tt, fam


# ------------------------------------------------------------------ training

def he_init(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM, dtype=np.float32)
    o = 0
    p[o:o + H * F] = rng.normal(0, math.sqrt(2.0 / F), H * F); o += H * F + H
    p[o:o + H * H] = rng.normal(0, math.sqrt(2.0 / H), H * H); o += H * H + H
    p[o:o + O * H] = rng.normal(0, math.sqrt(2.0 / H), O * H)
    return p


def train(X: np.ndarray, times: np.ndarray, epochs: int = 4000, lr: float = 3e-3, seed: int = 0):
    """Standardise, then train on the GPU (full batch Adam); returns the model dict."""
    import torch
    L = _lib()
    Y = np.log(times)
    xm, xs = X.mean(0), X.std(0)
    xs[xs == 0] = 1.0
    ym, ys = Y.mean(0), Y.std(0)
    ys[ys == 0] = 1.0
    Xs = ((X - xm) / xs).astype(np.float32)
    Ys = ((Y - ym) / ys).astype(np.float32)
    p = torch.from_numpy(he_init(seed)).cuda()
    Xd = torch.from_numpy(Xs).cuda()
    Yd = torch.from_numpy(Ys).cuda()
    m = torch.zeros(NPARAM, device="cuda")
    v = torch.zeros(NPARAM, device="cuda")
    hist = torch.zeros(epochs, device="cuda")
    code = L.rst_mlp_train(ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(Xd.data_ptr()),
                           ctypes.c_void_p(Yd.data_ptr()), len(Xs), epochs, lr, ctypes.c_void_p(m.data_ptr()),
                           ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(hist.data_ptr()), _stream())
    _check("rst_mlp_train", code)
    return {"params": p.cpu().numpy().tolist(),
            "norm": [*xm.tolist(), *xs.tolist(), *ym.tolist(), *ys.tolist()],
            "margin": 0.0, "epochs": epochs, "lr": lr, "seed": seed,
            "loss_first": float(hist[0].item()), "loss_last": float(hist[-1].item())}


def predict(X: np.ndarray):
    """The loaded network on the GPU (rst_selector_predict) for raw feature
    rows X: (predicted natural-log times [B][3], chosen STRATS index [B])."""
    import torch
    L = _lib()
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    B = Xd.shape[0]
    pred = torch.empty((B, O), dtype=torch.float32, device="cuda")
    choice = torch.empty(B, dtype=torch.int32, device="cuda")
    _check("rst_selector_predict", L.rst_selector_predict(ctypes.c_void_p(Xd.data_ptr()), B,
                                                          ctypes.c_void_p(pred.data_ptr()),
                                                          ctypes.c_void_p(choice.data_ptr()), _stream()))
    idx = np.array([CHOICE_INDEX[int(c)] for c in choice.cpu().numpy()], dtype=np.int64)
    return pred.cpu().numpy(), idx


def load_into_library(model: dict) -> None:
    L = _lib()
    p = np.ascontiguousarray(np.asarray(model["params"], dtype=np.float32))
    norm = np.ascontiguousarray(np.asarray(model["norm"], dtype=np.float32))
    _check("rst_selector_load", L.rst_selector_load(p.ctypes.data, norm.ctypes.data, float(model["margin"])))


def load_default() -> dict | None:
    if not os.path.exists(WEIGHTS_PATH):
        return None
    with open(WEIGHTS_PATH) as fh:
        model = json.load(fh)
    load_into_library(model)
    return model


def select(off, col, root: int):
    """(strategy name, predicted log-times) for one device-resident graph."""
    import torch
    L = _lib()
    choice = ctypes.c_int(0)
    pred = np.zeros(O, dtype=np.float32)
    bits = 64 if off.dtype == torch.int64 else 32
    code = L.rst_select(ctypes.c_void_p(off.data_ptr()), bits, ctypes.c_void_p(col.data_ptr()), off.numel() - 1,
                        col.numel(), int(root), ctypes.byref(choice), pred.ctypes.data, _stream())
    _check("rst_select", code)
    return STRATS[CHOICE_INDEX[choice.value]], pred
