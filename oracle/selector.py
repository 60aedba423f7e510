"""Double-precision oracle of the strategy selector (TEST INFRASTRUCTURE ONLY).

* ``features``: the 12 selector features from exact integer statistics of the
  CSR (degree moments, an 8-level BFS probe from the root, round-1 hook
  components and the edges that survive that hook pass), following the
  definitions stated in include/rst.h.
* ``forward`` / ``loss_grad`` / ``adam_step``: the 12-64-64-3 ReLU network,
  its mean-squared-error loss and gradient (ReLU'(0) = 0), and one Adam step
  (Kingma & Ba 2015), all in float64.
* ``predict`` / ``choose`` / ``regret``: the loaded model's float64 inference
  (standardise, forward, un-standardise), the strategy choice with the
  fallback margin, and the mean regret over graphs -- the checkers of the
  library's on-device inference and of the selector's evaluation.

Pins (tests/test_selector.py): central finite differences of ``loss_grad``,
the closed form of a first Adam step, hand-computed features of small graphs
(round-1 components and surviving edges of a hand-derived case), round-1
components against a plain union-find, the choice rule on hand-built
predictions.
"""
from __future__ import annotations

import numpy as np

F, H, O = 12, 64, 3
W1, B1 = 0, H * F
W2 = B1 + H
B2 = W2 + H * H
W3 = B2 + H
B3 = W3 + O * H
NPARAM = B3 + O   # 5187


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[W1:B1].reshape(H, F), p[B1:W2], p[W2:B2].reshape(H, H), p[B2:W3],
            p[W3:B3].reshape(O, H), p[B3:NPARAM])


def forward(p, X):
    w1, b1, w2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss_grad(p, X, T):
    """L = mean over batch and outputs of (y - t)^2, and dL/dp (float64)."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    d = y - T
    loss = float(np.sum(d * d) / (B * O))
    dy = 2.0 * d / (B * O)
    g = np.zeros(NPARAM)
    g[W3:B3] = (dy.T @ h2).ravel()
    g[B3:NPARAM] = dy.sum(0)
    dh2 = (dy @ w3) * (z2 > 0)
    g[W2:B2] = (dh2.T @ h1).ravel()
    g[B2:W3] = dh2.sum(0)
    dh1 = (dh2 @ w2) * (z1 > 0)
    g[W1:B1] = (dh1.T @ X).ravel()
    g[B1:W2] = dh1.sum(0)
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def he_init(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM)
    p[W1:B1] = rng.normal(0, np.sqrt(2.0 / F), H * F)
    p[W2:B2] = rng.normal(0, np.sqrt(2.0 / H), H * H)
    p[W3:B3] = rng.normal(0, np.sqrt(2.0 / H), O * H)
    return p


# ------------------------------------------------------------------ features

def _probe(n, off, col, root, max_levels=8):
    level = np.full(n, -1, dtype=np.int64)
    level[root] = 0
    frontier = np.array([root], dtype=np.int64)
    sizes = []
    finished = False
    L = 0
    while True:
        sizes.append(len(frontier))
        if L + 1 >= max_levels:
            break
        if len(frontier) == 0:
            break
        starts, ends = off[frontier], off[frontier + 1]
        idx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]) if len(frontier) else np.array([], np.int64)
        nb = np.unique(col[idx]) if len(idx) else np.array([], np.int64)
        nb = nb[level[nb] < 0]
        level[nb] = L + 1
        frontier = nb
        L += 1
        if len(frontier) == 0:
            finished = True
            break
    return sizes, finished


def first_neighbours(n, off, col):
    """first[u] = the first entry of u's sorted row other than u (-1: none)."""
    off = np.asarray(off, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    d = np.diff(off)
    src = np.repeat(np.arange(n, dtype=np.int64), d)
    idx = np.flatnonzero(col != src)
    first = np.full(n, -1, dtype=np.int64)
    rows, at = np.unique(src[idx], return_index=True)
    first[rows] = col[idx[at]]
    return first


def round1_components(n, first):
    """Component of every vertex in the graph of the round-1 hooks {u, first[u]}
    (connected components of that graph; isolated vertices alone)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    u = np.flatnonzero(first >= 0)
    a = coo_matrix((np.ones(len(u)), (u, first[u])), shape=(n, n))
    return connected_components(a, directed=False)[1]


def features(n, offsets, cols, root):
    off = np.asarray(offsets, dtype=np.int64)
    col = np.asarray(cols, dtype=np.int64)
    A = int(off[n])
    d = np.diff(off).astype(np.int64)
    N = float(n)
    s1, s2, s3 = float(d.sum()), float((d * d).sum()), float((d * d * d).sum())
    mu = s1 / N
    var = s2 / N - mu * mu
    sd = np.sqrt(var) if var > 0 else 0.0
    m3 = s3 / N - 3 * mu * (s2 / N) + 2 * mu ** 3
    m = A // 2
    f = np.zeros(F)
    f[0] = np.log2(N)
    f[1] = np.log2(max(m, 1))
    f[2] = mu
    f[3] = sd / mu if mu > 0 else 0.0
    f[4] = m3 / sd ** 3 if sd > 0 else 0.0
    f[5] = np.log2(1.0 + d.max()) if n else 0.0
    f[6] = float((d <= 2).sum()) / N
    if d[root] == 0:
        sizes, finished = [], True
        reached = 1.0
    else:
        sizes, finished = _probe(n, off, col, root)
        # the probe's frontiers are the BFS levels 0..levels-1 (the final empty one excluded)
        if finished and sizes and sizes[-1] == 0:
            sizes = sizes[:-1]
        reached = float(sum(sizes))
    levels = len(sizes)
    f[7] = np.log2(1.0 + reached)
    f3 = float(sizes[3]) if levels > 3 else 0.0
    f7 = float(sizes[7]) if levels > 7 else 0.0
    f[8] = np.log2((1.0 + f7) / (1.0 + f3))
    if levels == 0 or finished:
        ecc = float(levels if levels > 0 else 1)
    else:
        rest = N - reached
        fr = float(sizes[-1] if sizes[-1] > 0 else 1)
        ecc = levels + (rest / fr if rest > 0 else 0.0)
    f[9] = np.log2(1.0 + ecc)
    # round 1 of the min-key hooking: every vertex hooks along its first
    # neighbour other than itself (the smallest key, rows being sorted)
    first = first_neighbours(n, off, col)
    u = np.arange(n)
    ok = first >= 0
    mutual = np.zeros(n, bool)
    mutual[ok] = first[first[ok]] == u[ok]
    c1 = int((mutual & ok & (u < first)).sum())   # components with edges: one mutual pair each
    f[10] = np.log2(max(c1, 1) / N)
    comp = round1_components(n, first)
    src = np.repeat(np.arange(n, dtype=np.int64), d)
    keep = src < col
    f[11] = float((comp[src[keep]] != comp[col[keep]]).sum()) / m if m > 0 else 0.0
    return f


# ------------------------------------------------------------------ inference and evaluation

def predict(params, norm, X):
    """Predicted natural-log times of the model (params, norm = feature means,
    feature stds, target means, target stds) for raw feature rows X."""
    norm = np.asarray(norm, dtype=np.float64)
    xm, xs, ym, ys = norm[:F], norm[F:2 * F], norm[2 * F:2 * F + O], norm[2 * F + O:]
    xs = np.where(xs > 0, xs, 1.0)
    ys = np.where(ys > 0, ys, 1.0)
    y, _ = forward(params, (np.asarray(X, dtype=np.float64) - xm) / xs)
    return y * ys + ym


def choose(pred, margin):
    """Index of the chosen strategy per row (0 BFS, 1 CC+Euler, 2 PR-RST): the
    smallest prediction (the first on ties), replaced by CC+Euler when it
    beats CC+Euler's prediction by less than the margin."""
    pred = np.asarray(pred, dtype=np.float64)
    out = np.empty(len(pred), dtype=np.int64)
    for i, p in enumerate(pred):
        best = 1
        for k in range(O):
            if p[k] < p[best]:
                best = k
        if best != 1 and p[1] - p[best] < margin:
            best = 1
        out[i] = best
    return out


def regret(times, choice):
    """Mean over graphs of (t_chosen - t_best) / t_best."""
    times = np.asarray(times, dtype=np.float64)
    tb = times.min(1)
    tc = times[np.arange(len(times)), np.asarray(choice)]
    return float(np.mean((tc - tb) / tb))
