"""rst_bcc (Tarjan-Vishkin on the Euler tour) against the Hopcroft-Tarjan
oracle: block label of every arc, cut vertices and block count, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(off_np, col_np, n):
    import paper_2603_11645_gb300 as rst
    off = torch.from_numpy(np.ascontiguousarray(off_np)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(col_np)).cuda()
    lab, cut, nb = rst.bcc(off, col)
    return lab.cpu().numpy().view(np.uint32), cut.cpu().numpy(), nb


def _check(n, off, col, name=""):
    lab, cut, nb = _run(off, col, n)
    wl, wc, wn = oracle.bcc(n, off, col)
    assert nb == wn, name
    assert np.array_equal(lab, wl), name
    assert np.array_equal(cut, wc), name


def _multigraph(n, edges):
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        rows[v].append(u)
    off = np.zeros(n + 1, dtype=np.int32)
    for i in range(n):
        rows[i].sort()
        off[i + 1] = off[i] + len(rows[i])
    return off, np.array([w for r in rows for w in r] or [0], dtype=np.int32)[:off[n]]


def test_bcc_small_families():
    from test_gpu_parity import edge_cases, small_graphs
    for g in small_graphs() + edge_cases():
        _check(g.n, g.offsets, g.cols, g.name)


@pytest.mark.parametrize("seed", range(12))
def test_bcc_random_multigraphs_with_loops(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 300))
    m = int(rng.integers(0, 3 * n))
    edges = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
    off, col = _multigraph(n, edges)
    _check(n, off, col, f"multigraph seed {seed}")


@pytest.mark.parametrize("which", ["trees", "cactus", "sparse_er", "chords"])
def test_bcc_many_blocks(which):
    rng = np.random.default_rng(7)
    if which == "trees":      # a forest: every edge a bridge
        n = 5000
        par = [int(rng.integers(0, max(v, 1))) for v in range(n)]
        g = graphs.from_edges(n, list(range(1, n)), par[1:], root=0)
    elif which == "cactus":   # cycles hanging off cycles: many blocks and cut vertices
        edges, n = [], 1
        for _ in range(800):
            a = int(rng.integers(0, n))
            k = int(rng.integers(2, 7))
            cyc = [a] + list(range(n, n + k))
            n += k
            edges += [(cyc[i], cyc[(i + 1) % len(cyc)]) for i in range(len(cyc))]
        g = graphs.from_edges(n, [e[0] for e in edges], [e[1] for e in edges], root=0)
    elif which == "sparse_er":
        g = graphs.erdos_renyi(20000, 14000, seed=8)
    else:
        g = graphs.chain_chords(30000, 0.002, seed=9)
    _check(g.n, g.offsets, g.cols, which)


@pytest.mark.parametrize("which", ["grid1024", "rmat18", "grid4096"])
def test_bcc_large(which):
    g = {"grid1024": lambda: graphs.grid(1024, 1024, seed=5, permute=True),
         "rmat18": lambda: graphs.rmat(18, 8, seed=6, connect=False, offsets_bits=64),
         "grid4096": graphs.workload_grid4096}[which]()
    _check(g.n, g.offsets, g.cols, which)
