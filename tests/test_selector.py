"""Strategy selector: oracle pins (CPU), GPU kernels against the oracle, and
the trained network's regret on held-out graphs."""
import json
import math
import os

import numpy as np
import pytest

from oracle import selector as OS
from paper_2603_11645_gb300 import graphs


def _batch(seed, B=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, OS.F))
    T = rng.normal(size=(B, OS.O))
    p = OS.he_init(seed) + rng.normal(0, 0.05, OS.NPARAM)
    return p, X, T


# ------------------------------------------------------------------ oracle pins

def test_oracle_gradient_matches_finite_differences():
    p, X, T = _batch(1)
    loss, g = OS.loss_grad(p, X, T)
    rng = np.random.default_rng(2)
    idx = rng.choice(OS.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(OS.NPARAM)
        e[i] = h
        fd = (OS.loss_grad(p + e, X, T)[0] - OS.loss_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_oracle_adam_first_step_closed_form():
    # with m = v = 0 at t = 1 the bias-corrected moments are g and g^2, so the
    # step is lr * g / (|g| + eps)
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    q, m, v = OS.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_oracle_features_of_a_path():
    n = 10
    g = graphs.from_edges(n, list(range(n - 1)), list(range(1, n)), root=0)
    f = OS.features(n, g.offsets, g.cols, 0)
    mu = 18 / 10
    var = (2 * 1 + 8 * 4) / 10 - mu * mu
    assert f[0] == pytest.approx(math.log2(10))
    assert f[1] == pytest.approx(math.log2(9))
    assert f[2] == pytest.approx(mu)
    assert f[3] == pytest.approx(math.sqrt(var) / mu)
    assert f[5] == pytest.approx(math.log2(3))
    assert f[6] == pytest.approx(1.0)
    # probe: levels 0..7 hold one vertex each, not finished after 8 levels
    assert f[7] == pytest.approx(math.log2(9))
    assert f[8] == pytest.approx(0.0)
    assert f[9] == pytest.approx(math.log2(1 + 8 + 2 / 1))
    # round 1: only 0 and 1 choose each other, and every vertex joins them
    # (u hooks along u - 1), so no edge survives
    assert f[10] == pytest.approx(math.log2(1 / 10))
    assert f[11] == pytest.approx(0.0)


def test_oracle_features_of_a_star():
    n = 9
    g = graphs.from_edges(n, [0] * 8, list(range(1, n)), root=3)
    f = OS.features(n, g.offsets, g.cols, 3)
    # levels: {3}, {0}, {1,2,4,...,8}; finished after 3 levels
    assert f[7] == pytest.approx(math.log2(10))
    assert f[9] == pytest.approx(math.log2(1 + 3))
    # every leaf's first neighbour is 0, 0's first neighbour is 1: one mutual
    # pair, one round-1 component, no surviving edge
    assert f[10] == pytest.approx(math.log2(1 / 9))
    assert f[11] == pytest.approx(0.0)


def test_oracle_round1_of_a_hand_derived_case():
    """Edges 0-2, 1-3, 2-3: rows 0:[2] 1:[3] 2:[0,3] 3:[1,2], so the first
    neighbours are 0->2, 1->3, 2->0, 3->1: two mutual pairs, round-1
    components {0,2} and {1,3}, and the edge 2-3 (one of three) survives."""
    g = graphs.from_edges(4, [0, 1, 2], [2, 3, 3], root=0)
    f = OS.features(4, g.offsets, g.cols, 0)
    assert f[10] == pytest.approx(math.log2(2 / 4))
    assert f[11] == pytest.approx(1 / 3)
    first = OS.first_neighbours(4, g.offsets, g.cols)
    assert list(first) == [2, 3, 0, 1]


def _components_by_union_find(n, first):
    par = list(range(n))

    def find(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x
    for u in range(n):
        if first[u] >= 0:
            a, b = find(u), find(int(first[u]))
            if a != b:
                par[max(a, b)] = min(a, b)
    return [find(u) for u in range(n)]


def test_oracle_round1_components_against_union_find():
    """The first neighbour skips self-loops and the components of the hook
    graph equal a plain union-find's, on multigraphs with loops and repeats."""
    rng = np.random.default_rng(5)
    for t in range(30):
        n = int(rng.integers(1, 40))
        k = int(rng.integers(0, 3 * n))
        u = rng.integers(0, n, k)
        v = np.where(rng.random(k) < 0.15, u, rng.integers(0, n, k))  # some self-loops
        src = np.concatenate([u, v])
        dst = np.concatenate([v, u])
        order = np.lexsort((dst, src))
        src, dst = src[order], dst[order]
        off = np.zeros(n + 1, dtype=np.int64)
        np.add.at(off, src + 1, 1)
        off = np.cumsum(off)
        first = OS.first_neighbours(n, off, dst)
        for x in range(n):
            row = [int(c) for c in dst[off[x]:off[x + 1]] if c != x]
            assert first[x] == (row[0] if row else -1)
        comp = OS.round1_components(n, first)
        uf = _components_by_union_find(n, first)
        for a in range(n):
            for b in range(n):
                assert (comp[a] == comp[b]) == (uf[a] == uf[b])


def test_oracle_choice_rule():
    """Smallest predicted log-time wins; CC+Euler (index 1) is kept when the
    winner's predicted gain over it is below the margin."""
    pred = np.array([[0.0, 1.0, 2.0],    # BFS by 1.0
                     [3.0, 1.0, 0.95],   # PR-RST by 0.05
                     [5.0, 1.0, 5.0],    # CC+Euler
                     [1.0, 1.0, 2.0]])   # tie: CC+Euler (the first smallest from index 1 stays)
    assert list(OS.choose(pred, 0.0)) == [0, 2, 1, 1]
    assert list(OS.choose(pred, 0.1)) == [0, 1, 1, 1]
    assert list(OS.choose(pred, 2.0)) == [1, 1, 1, 1]
    t = np.array([[1.0, 2.0, 4.0], [2.0, 1.0, 1.0]])
    assert OS.regret(t, [0, 1]) == pytest.approx(0.0)
    assert OS.regret(t, [1, 2]) == pytest.approx(0.5)


# ------------------------------------------------------------------ GPU kernels vs oracle

torch = pytest.importorskip("torch")


def _multigraph(n, k, seed):
    """A CSR with self-loops and repeated arcs (rows sorted, symmetric)."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, k)
    v = np.where(rng.random(k) < 0.1, u, rng.integers(0, n, k))
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    g = graphs.Graph(f"multi{n}", n, np.cumsum(off).astype(np.int32), dst.astype(np.int32),
                     int(rng.integers(0, n)))
    return g


@pytest.mark.gpu
def test_gpu_features_match_oracle():
    from paper_2603_11645_gb300 import selector as S
    cases = [graphs.grid(40, 30, seed=1, root="random"), graphs.chain_chords(5000, 0.001, seed=2),
             graphs.rmat(12, 16, seed=3, connect=True, offsets_bits=32), graphs.random_4regular(3000, seed=4),
             graphs.erdos_renyi(2000, 1500, seed=5), graphs.from_edges(5, [0, 1], [1, 2], root=4),
             graphs.from_edges(4, [0, 1, 2], [2, 3, 3], root=1),
             graphs.rmat(16, 16, seed=6, connect=True, offsets_bits=64),
             _multigraph(6000, 15000, 7)]
    for g in cases:
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        got = S.features(off, col, g.root)
        want = OS.features(g.n, g.offsets, g.cols, g.root)
        assert np.allclose(got, want, rtol=2e-6, atol=2e-6), (g.name, got, want)


@pytest.mark.gpu
def test_gpu_mlp_matches_oracle():
    import ctypes
    from paper_2603_11645_gb300 import selector as S
    L = S._lib()
    p, X, T = _batch(7, B=513)
    pd = torch.tensor(p, dtype=torch.float32, device="cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    Y = torch.zeros(513, 3, device="cuda")
    S._check("fwd", L.rst_mlp_forward(ctypes.c_void_p(pd.data_ptr()), ctypes.c_void_p(Xd.data_ptr()), 513,
                                      ctypes.c_void_p(Y.data_ptr()), S._stream()))
    y_ref, _ = OS.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.allclose(Y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4)
    G = torch.zeros(OS.NPARAM, device="cuda")
    loss = torch.zeros(1, device="cuda")
    S._check("grad", L.rst_mlp_loss_grad(ctypes.c_void_p(pd.data_ptr()), ctypes.c_void_p(Xd.data_ptr()),
                                         ctypes.c_void_p(Td.data_ptr()), 513, ctypes.c_void_p(G.data_ptr()),
                                         ctypes.c_void_p(loss.data_ptr()), S._stream()))
    l_ref, g_ref = OS.loss_grad(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                                T.astype(np.float32).astype(np.float64))
    g = G.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - l_ref) <= 1e-4 * abs(l_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # one Adam step
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    S._check("adam", L.rst_mlp_adam(ctypes.c_void_p(pd.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                    ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), OS.NPARAM, 1,
                                    1e-3, 0.9, 0.999, 1e-8, S._stream()))
    q_ref, _, _ = OS.adam_step(p.astype(np.float32).astype(np.float64), g, np.zeros(OS.NPARAM), np.zeros(OS.NPARAM),
                               1, lr=1e-3)
    assert np.allclose(pd.cpu().numpy(), q_ref, rtol=0, atol=2e-6)


@pytest.mark.gpu
def test_gpu_training_fits_a_smooth_target():
    from paper_2603_11645_gb300 import selector as S
    rng = np.random.default_rng(11)
    X = rng.normal(size=(800, 12))
    t = np.exp(np.stack([X[:, 0] + 0.5 * X[:, 1], np.sin(X[:, 2]), X[:, 3] * X[:, 4] * 0.3], 1))
    model = S.train(X, t, epochs=1500, lr=3e-3, seed=1)
    assert model["loss_last"] < 0.2 * model["loss_first"]


@pytest.mark.gpu
def test_gpu_inference_matches_oracle():
    """rst_selector_predict (standardise, network, margin choice on the GPU)
    against the oracle's float64 inference, for a random model and random
    feature rows; choices are compared where no near-tie can flip them."""
    from paper_2603_11645_gb300 import selector as S
    rng = np.random.default_rng(21)
    p = OS.he_init(3)
    norm = np.concatenate([rng.normal(size=OS.F), rng.uniform(0.5, 2.0, OS.F), rng.normal(size=OS.O),
                           rng.uniform(0.5, 2.0, OS.O)])
    X = rng.normal(size=(300, OS.F)) * 2
    for margin in (0.0, 0.3):
        S.load_into_library({"params": p.tolist(), "norm": norm.tolist(), "margin": margin})
        pred, idx = S.predict(X)
        p32 = p.astype(np.float32).astype(np.float64)
        n32 = norm.astype(np.float32).astype(np.float64)
        want = OS.predict(p32, n32, X.astype(np.float32).astype(np.float64))
        assert np.allclose(pred, want, rtol=1e-4, atol=1e-4)
        wc = OS.choose(want, margin)
        srt = np.sort(want, 1)
        gain = want[:, 1] - want.min(1)  # predicted gain of the best over CC+Euler
        near_margin = (gain > 0) & (np.abs(gain - margin) <= 1e-3)
        safe = (srt[:, 1] - srt[:, 0] > 1e-3) & ~near_margin
        assert safe.sum() > 250
        assert np.array_equal(idx[safe], wc[safe])
    S.load_default()


# ------------------------------------------------------------------ regret of the trained selector

def _trained():
    from paper_2603_11645_gb300 import selector as S
    if not os.path.exists(S.WEIGHTS_PATH):
        pytest.skip("no trained selector weights in the repository")
    with open(S.WEIGHTS_PATH) as fh:
        model = json.load(fh)
    data = os.path.join(os.path.dirname(S.__file__), "selector_data")
    ho = [f for f in os.listdir(data) if f.startswith("heldout_")] if os.path.isdir(data) else []
    if not ho:
        pytest.skip("no held-out timing data in the repository")
    return S, model, os.path.join(data, ho[0])


def test_stored_model_regret_by_the_oracle():
    """The committed network, evaluated by the oracle's float64 inference on
    the stored held-out features, beats always-CC+Euler and stays within 10%
    regret (a check of the stored weights and data, independent of the GPU)."""
    S, model, path = _trained()
    X, Tt, fam = S.load_dataset(path)
    sel = OS.choose(OS.predict(model["params"], model["norm"], X), model["margin"])
    r_sel = OS.regret(Tt, sel)
    assert r_sel <= OS.regret(Tt, np.ones(len(Tt), dtype=int))
    assert r_sel <= 0.10


@pytest.mark.gpu
def test_gpu_selector_regret_on_heldout_graphs():
    """What the network gains over the method without it: the GPU's own
    choices (rst_selector_predict on the held-out graphs' GPU features) score
    at most 10% mean regret against the exhaustively timed strategies, and
    less than always choosing CC+Euler."""
    S, model, path = _trained()
    X, Tt, fam = S.load_dataset(path)
    S.load_into_library(model)
    pred, sel = S.predict(X)
    r_sel = OS.regret(Tt, sel)
    r_cc = OS.regret(Tt, np.ones(len(Tt), dtype=int))
    assert r_sel <= r_cc
    assert r_sel <= 0.10


@pytest.mark.gpu
def test_rst_select_end_to_end_on_heldout_graphs():
    """rst_select on regenerated held-out graphs: its features equal the stored
    ones and its choice is the one the stored features give."""
    S, model, path = _trained()
    X, Tt, fam = S.load_dataset(path)
    S.load_into_library(model)
    _, stored_choice = S.predict(X)
    import csv
    with open(path) as fh:
        rows = list(csv.DictReader(fh))
    small = [i for i, r in enumerate(rows) if int(r["n"]) <= (1 << 18)][:8]
    assert small
    for i in small:
        g = S.family_graph(i, "heldout")
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        f = S.features(off, col, g.root)
        assert np.allclose(f, X[i], rtol=1e-5, atol=1e-5), (i, f, X[i])
        choice, pred = S.select(off, col, g.root)
        assert choice == S.STRATS[stored_choice[i]]


@pytest.mark.gpu
def test_auto_strategy_builds_what_the_selector_chooses():
    """RST_AUTO runs the strategy rst_select picks, with that strategy's exact result."""
    import oracle
    import paper_2603_11645_gb300 as rst
    from paper_2603_11645_gb300 import selector as S
    if S.load_default() is None:
        pytest.skip("no trained selector weights in the repository")
    cases = [graphs.grid(300, 200, seed=61, permute=True, root="random"),
             graphs.rmat(14, 16, seed=62, connect=True, offsets_bits=32),
             graphs.chain_chords(20000, 0.01, seed=63),
             graphs.random_4regular(5000, seed=64)]
    seen = set()
    for g in cases:
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        choice, pred = S.select(off, col, g.root)
        assert np.all(np.isfinite(pred))
        par = rst.build(off, col, g.root, "auto").cpu().numpy()
        if choice == "cc_euler":
            want = oracle.rst(g.n, g.offsets, g.cols, g.root)
        elif choice == "bfs":
            want = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
        else:
            want = oracle.prrst(g.n, g.offsets, g.cols, g.root)[0]
        assert np.array_equal(par, want), (g.name, choice)
        seen.add(choice)
    assert seen  # at least one strategy exercised through RST_AUTO
