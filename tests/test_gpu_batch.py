"""rst_build_batch (GPU) against the oracle graph by graph, and against
per-graph rst_build calls."""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_batch(seed=0, G=48):
    rng = np.random.default_rng(seed)
    gs = []
    for i in range(G):
        kind = i % 6
        n = int(rng.integers(50, 3000))
        if kind == 0:
            W = int(rng.integers(1, 60))
            gs.append(graphs.grid(W, max(1, n // W), seed=seed * 100 + i, root="random"))
        elif kind == 1:
            gs.append(graphs.chain_chords(n, float(rng.choice([0.0, 0.001, 0.05])), seed=seed * 100 + i))
        elif kind == 2:
            gs.append(graphs.rmat(int(rng.integers(6, 12)), 8, seed=seed * 100 + i, connect=bool(i % 4),
                                  offsets_bits=32))
        elif kind == 3:
            gs.append(graphs.erdos_renyi(n, int(n * rng.uniform(0.3, 1.5)), seed=seed * 100 + i))
        elif kind == 4:
            gs.append(graphs.from_edges(1, [], [], name="single", root=0))
        else:
            gs.append(graphs.from_edges(7, [0, 2, 4, 5], [1, 3, 5, 6], name="forest", root=int(rng.integers(0, 7))))
    return graphs.pack_batch(gs)


def to_dev(b):
    d = torch.device("cuda:0")
    return (torch.from_numpy(b.offsets).to(d), torch.from_numpy(b.cols).to(d),
            torch.from_numpy(b.vtx_off).to(d), torch.from_numpy(b.arc_off).to(d),
            torch.from_numpy(b.roots).to(d))


@pytest.mark.parametrize("strategy", ["cc_euler", "bfs"])
@pytest.mark.parametrize("seed", [0, 1])
def test_batch_matches_oracle_per_graph(strategy, seed):
    import paper_2603_11645_gb300 as rst
    b = small_batch(seed)
    par = rst.build_batch(*to_dev(b), strategy=strategy).cpu().numpy()
    for g_i, g in enumerate(b.graphs):
        got = par[b.vtx_off[g_i]:b.vtx_off[g_i + 1]]
        if strategy == "cc_euler":
            want = oracle.rst(g.n, g.offsets, g.cols, g.root)
        else:
            want = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
        assert np.array_equal(got, want), (g_i, g.name)


def test_batch_equals_single_calls():
    import paper_2603_11645_gb300 as rst
    b = small_batch(3, G=24)
    off, col, vo, ao, roots = to_dev(b)
    par = rst.build_batch(off, col, vo, ao, roots).cpu().numpy()
    for g_i, g in enumerate(b.graphs):
        o0 = int(b.vtx_off[g_i]) + g_i
        a0, a1 = int(b.arc_off[g_i]), int(b.arc_off[g_i + 1])
        single = rst.build(off[o0:o0 + g.n + 1].contiguous(), col[a0:a1].contiguous(), g.root).cpu().numpy()
        assert np.array_equal(par[b.vtx_off[g_i]:b.vtx_off[g_i + 1]], single)


def test_batch_workload_4096_graphs():
    """The mixed 4096-graph workload the benchmark times, checked graph by graph."""
    import paper_2603_11645_gb300 as rst
    b = graphs.workload_batch()
    par = rst.build_batch(*to_dev(b)).cpu().numpy()
    for g_i, g in enumerate(b.graphs):
        want = oracle.rst(g.n, g.offsets, g.cols, g.root)
        assert np.array_equal(par[b.vtx_off[g_i]:b.vtx_off[g_i + 1]], want), (g_i, g.name)


@pytest.mark.skipif(__import__("os").environ.get("RST_MAX_SIZE") != "1", reason="opt-in: RST_MAX_SIZE=1")
def test_batch_literal_size_law():
    """4,096 graphs with n log-uniform in [1K, 256K] (about 2.5e9 arcs, int64
    packed offsets): every graph's slice checked by the verifier on the GPU,
    64 of them against the oracle bit for bit."""
    import paper_2603_11645_gb300 as rst
    b = graphs.workload_batch(hi=262144)
    dev = to_dev(b)
    par = rst.build_batch(*dev)
    assert b.A > 2 ** 31
    parn = par.cpu().numpy()
    rng = np.random.default_rng(7)
    sample = set(rng.choice(b.G, 64, replace=False).tolist())
    for g_i, g in enumerate(b.graphs):
        sl = parn[b.vtx_off[g_i]:b.vtx_off[g_i + 1]]
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        assert rst.verify(off, col, g.root, torch.from_numpy(sl.copy()).cuda()) == 0, g_i
        if g_i in sample:
            assert np.array_equal(sl, oracle.rst(g.n, g.offsets, g.cols, g.root)), (g_i, g.name)
