"""CC+Euler's list build around a giant round-1 component (GPU).

When one round-1 component holds most vertices (power-law graphs: a hub's
neighbourhood merges in round 1), the contracted edge list is built from the
rows of the vertices outside it only; an edge between such a vertex and the
giant whose smaller end lies in the giant takes its key from a search of
that end's row.  The list holds the same edges either way, so the forest,
the labels and the parents are the oracle's whichever path runs.  Each case
runs with the path forced (giant_share_pct 0), at the default share and
switched off (101), and is compared with the oracle bit for bit.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPARSE_STAT = 9  # rows read outside the giant (-1: every row)


def _stats():
    import paper_2603_11645_gb300 as rst
    L = rst.lib()
    L.rst_last_stats.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.rst_last_stats.restype = ctypes.c_int
    st = (ctypes.c_longlong * 10)()
    assert L.rst_last_stats(st, 10) == 10
    return list(st)


def _csr(n, u, v, offsets_bits=32):
    """Symmetric CSR with sorted rows, keeping repeated arcs and self-loops."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off).astype(np.int32 if offsets_bits == 32 else np.int64)
    return graphs.Graph("csr", n, off, np.ascontiguousarray(dst.astype(np.int32)), 0, {})


def star_and_pairs():
    """A star on 0 (leaves 1..9999 and 15000..15999) and 4,000 separate pairs
    {10000+k, 20000+k}; the larger end of every pair also meets the leaf
    15000 + k % 1000, which lies in the giant and below it, so that edge's
    key comes from a search of the leaf's row.  58% of the vertices are in
    the giant."""
    leaves = np.concatenate([np.arange(1, 10000), np.arange(15000, 16000)])
    k = np.arange(4000)
    u = np.concatenate([np.zeros(leaves.size, np.int64), 10000 + k, 20000 + k])
    v = np.concatenate([leaves, 20000 + k, 15000 + k % 1000])
    g = _csr(24000, u, v)
    g.root = 20017
    g.name = "star-and-pairs"
    return g


def multigraph(seed):
    """A giant (every vertex of [0, n/2) joined to 0, doubled) plus random
    edges with duplicates and self-loops over all vertices."""
    rng = np.random.default_rng(4100 + seed)
    n = int(rng.integers(500, 8000))
    h = n // 2
    a = np.arange(1, h)
    m = int(rng.integers(n // 4, 2 * n))
    ru = rng.integers(0, n, size=m)
    rv = rng.integers(0, n, size=m)
    rv = np.where(rng.random(m) < 0.05, ru, rv)  # self-loops
    u = np.concatenate([np.zeros(2 * a.size, np.int64), ru, ru[: m // 8]])
    v = np.concatenate([a, a, rv, rv[: m // 8]])  # repeated arcs
    g = _csr(n, u, v, offsets_bits=64 if seed % 2 else 32)
    g.root = int(rng.integers(0, n))
    g.name = f"multigraph-{seed}"
    return g


def _cases():
    return [
        graphs.rmat(14, 16, seed=41, connect=True, offsets_bits=64),
        graphs.rmat(13, 8, seed=42, connect=False),
        star_and_pairs(),
        multigraph(0),
        multigraph(1),
        multigraph(2),
        graphs.grid(120, 90, seed=43, permute=True, root="random"),
        graphs.erdos_renyi(20000, 30000, seed=44),
    ]


_CASES = None


def _case(i):
    global _CASES
    if _CASES is None:
        _CASES = _cases()
    return _CASES[i]


@pytest.fixture
def share():
    import paper_2603_11645_gb300 as rst
    yield rst.set_option
    rst.set_option("giant_share_pct", 75)


@pytest.mark.parametrize("pct", [0, 75, 101])
@pytest.mark.parametrize("ci", range(8))
def test_list_build_paths_match_oracle(ci, pct, share):
    import paper_2603_11645_gb300 as rst
    g = _case(ci)
    share("giant_share_pct", pct)
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    sparse = _stats()[SPARSE_STAT]
    assert np.array_equal(par, oracle.rst(g.n, g.offsets, g.cols, g.root)), (g.name, pct)
    if pct == 101:
        assert sparse == -1
    if pct == 0 and g.A > 0:
        assert 0 <= sparse < g.n  # forced: the largest sampled component's complement
    labels, uv, T = rst.cc(off, col)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert np.array_equal(labels.cpu().numpy(), lab), (g.name, pct)
    assert T == len(tu)
    got = uv.cpu().numpy()
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    assert np.array_equal(got[:, 0], tu) and np.array_equal(got[:, 1], tv), (g.name, pct)


def test_default_share_picks_the_path():
    """R-MAT (a hub merges most vertices in round 1) reads only the rows
    outside its giant; a permuted grid (round-1 components of a few vertices)
    and the star with 58% of its vertices in the giant read every row."""
    import paper_2603_11645_gb300 as rst
    rst.set_option("giant_share_pct", 75)
    for ci, want_sparse in [(0, True), (2, False), (6, False)]:
        g = _case(ci)
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        rst.build(off, col, g.root, "cc_euler")
        sparse = _stats()[SPARSE_STAT]
        if want_sparse:
            assert 0 <= sparse < g.n // 4, g.name
        else:
            assert sparse == -1, g.name
