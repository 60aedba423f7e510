"""Learned strategy selector: data generation, GPU training, evaluation.

The library's own timings of BFS, CC+Euler and PR-RST on seeded graphs train a
12-64-64-3 network (rst_mlp_train: forward, backward and Adam kernels on the
GPU) that predicts each strategy's log-time from 12 cheap features
(rst_selector_features).  rst_select / rst_build(RST_AUTO) pick the smallest
prediction and fall back to CC+Euler when the predicted gain is below a margin.

Graph families (seeded; training seeds 5000+i, held-out seeds 9000+i):
grids with aspect ratio log-uniform in [1, 4096], paths with uniformly random
chords at density log-uniform in [1e-6, 1e-1], R-MAT graphs connected to
vertex 0, and random 4-regular graphs; vertex counts log-uniform in
[2^14, 2^20].  BFS runs are capped at BFS_LEVEL_CAP levels; a capped run is
labelled with the time spent up to the cap (a lower bound that is never the
fastest strategy, so regret stays exact).
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
BFS_LEVEL_CAP = 4096
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")
FEATURE_NAMES = ["log2_n", "log2_m", "mean_deg", "deg_cv", "deg_skew", "log2_maxdeg", "frac_deg_le2",
                 "log2_probe_reached", "log2_probe_growth", "log2_ecc_est", "log2_r1_comp_frac",
                 "probe_reach_frac"]


def _lib():
    from . import lib
    L = lib()
    P, I, I32, I64, Fl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    L.rst_selector_features.argtypes = [P, I, P, I64, I64, I32, P, P]
    L.rst_selector_load.argtypes = [P, P, Fl]
    L.rst_select.argtypes = [P, I, P, I64, I64, I32, P, P, P]
    L.rst_mlp_forward.argtypes = [P, P, I, P, P]
    L.rst_mlp_loss_grad.argtypes = [P, P, P, I, P, P, P]
    L.rst_mlp_adam.argtypes = [P, P, P, P, I, I, Fl, Fl, Fl, Fl, P]
    L.rst_mlp_train.argtypes = [P, P, P, I, I, Fl, P, P, P, P]
    L.rst_set_option.argtypes = [ctypes.c_char_p, ctypes.c_longlong]
    for fn in ("rst_selector_features", "rst_selector_load", "rst_select", "rst_mlp_forward",
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
    n = int(round(math.exp(math.log(2 ** 14) + r[0] * (math.log(2 ** 20) - math.log(2 ** 14)))))
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
        scale = max(14, min(20, int(round(math.log2(n)))))
        g = graphs.rmat(scale, 16, seed=seed, connect=True, offsets_bits=32)
    else:
        g = graphs.random_4regular(max(n, 5), seed=seed)
    g.meta["split"] = split
    g.meta["index"] = i
    return g


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


def generate_dataset(split: str, count: int, path: str, reps: int = 3, log_every: int = 50):
    """Features and timings of `count` graphs of the split, written as CSV."""
    import torch
    rows = []
    t0 = time.time()
    for i in range(count):
        g = family_graph(i, split)
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        f = features(off, col, g.root)
        ts, cens = time_strategies(off, col, g.root, reps)
        rows.append([split, i, g.meta.get("family", "?"), g.n, g.m] + [float(x) for x in f] + ts + [int(cens)])
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


def predict_host(model: dict, X: np.ndarray) -> np.ndarray:
    """Predicted natural-log times (float64 host evaluation of the model)."""
    p = np.asarray(model["params"], dtype=np.float64)
    norm = np.asarray(model["norm"], dtype=np.float64)
    xm, xs, ym, ys = norm[:F], norm[F:2 * F], norm[2 * F:2 * F + O], norm[2 * F + O:]
    Xs = (X - xm) / xs
    o = 0
    w1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    w2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + O * H].reshape(O, H); o += O * H
    b3 = p[o:o + O]
    h1 = np.maximum(Xs @ w1.T + b1, 0)
    h2 = np.maximum(h1 @ w2.T + b2, 0)
    return (h2 @ w3.T + b3) * ys + ym


def choose(pred: np.ndarray, margin: float) -> np.ndarray:
    best = pred.argmin(1)
    cc = 1
    fallback = (best != cc) & (pred[:, cc] - pred[np.arange(len(pred)), best] < margin)
    best[fallback] = cc
    return best


def regret(times: np.ndarray, choice: np.ndarray) -> float:
    """Mean over graphs of (t_chosen - t_best) / t_best."""
    tb = times.min(1)
    tc = times[np.arange(len(times)), choice]
    return float(np.mean((tc - tb) / tb))


def fit_margin(model: dict, X: np.ndarray, times: np.ndarray) -> float:
    pred = predict_host(model, X)
    best_m, best_r = 0.0, None
    for mg in [0.0, 0.05, 0.1, 0.2, 0.3, 0.5, 0.75, 1.0]:
        r = regret(times, choose(pred, mg))
        if best_r is None or r < best_r - 1e-12:
            best_m, best_r = mg, r
    return best_m


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
    return {1: "bfs", 2: "cc_euler", 3: "pr_rst"}[choice.value], pred
