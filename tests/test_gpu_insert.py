"""rst_insert_edges (PR-RST rounds from an existing forest) against the
oracle's rounds from the same forest: bit-exact parent arrays."""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _graph(n, edges):
    return graphs.from_edges(n, [e[0] for e in edges], [e[1] for e in edges], root=0)


def _gpu_insert(init, new, root, canonical=False):
    import paper_2603_11645_gb300 as rst
    par = torch.from_numpy(np.asarray(init, dtype=np.int32)).cuda()
    uv = torch.from_numpy(np.asarray(new, dtype=np.int32).reshape(-1, 2)).cuda()
    rst.insert_edges(par, uv, root, canonical=canonical)
    return par.cpu().numpy()


@pytest.mark.parametrize("n,old,init,new,root", [
    (4, [(0, 1), (1, 2)], [0, 0, 1, 3], [(2, 3)], 0),
    (5, [(0, 1), (1, 2), (3, 4)], [0, 0, 1, 3, 3], [(4, 1)], 0),
    (5, [(0, 1), (1, 2), (3, 4)], [0, 0, 1, 3, 3], [(4, 1)], 4),
    (7, [(0, 5), (1, 6)], [0, 0, 2, 3, 4, 0, 1], [(5, 6), (0, 1)], 0),
    (3, [(0, 1)], [0, 0, 2], [], 2),                 # no insertion: re-rooting only
    (3, [(0, 1)], [0, 0, 2], [(2, 2), (0, 1)], 0),   # self-loop and an edge inside a tree
])
def test_insert_small(n, old, init, new, root):
    g = _graph(n, old + new)
    want, _ = oracle.prrst(n, g.offsets, g.cols, root, init=init)
    assert np.array_equal(_gpu_insert(init, new, root), want)


def _dropped(g, frac, seed):
    """g minus a random fraction of its edges, and the dropped edges."""
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets)).astype(np.int64)
    col = g.cols.astype(np.int64)
    lo, hi = np.minimum(src, col), np.maximum(src, col)
    h = (lo * 0x9E3779B1 + hi * 0x85EBCA77 + seed) % 1000003
    drop = h < frac * 1000003
    keep = ~drop
    g0 = graphs.from_edges(g.n, src[keep & (src < col)], col[keep & (src < col)], root=g.root)
    new = np.stack([src[drop & (src < col)], col[drop & (src < col)]], 1)
    return g0, new[rng.permutation(len(new))]


@pytest.mark.parametrize("which,frac", [("er", 0.3), ("grid", 0.25), ("rmat", 0.5), ("chain", 0.2)])
def test_insert_random_batches(which, frac):
    g = {"er": lambda: graphs.erdos_renyi(20000, 25000, seed=51),
         "grid": lambda: graphs.grid(300, 200, seed=52, permute=True, root="random"),
         "rmat": lambda: graphs.rmat(14, 8, seed=53, connect=False, offsets_bits=32),
         "chain": lambda: graphs.chain_chords(30000, 0.001, seed=54)}[which]()
    g0, new = _dropped(g, frac, seed=5)
    init = oracle.rst(g0.n, g0.offsets, g0.cols, g0.root)
    root = int(g.root)
    want, _ = oracle.prrst(g.n, g.offsets, g.cols, root, init=init)
    got = _gpu_insert(init, new, root)
    assert np.array_equal(got, want)
    assert oracle.verify(g.n, g.offsets, g.cols, root, got) == oracle.VALID


def test_insert_after_a_gpu_build():
    import paper_2603_11645_gb300 as rst
    g = graphs.grid(1024, 1024, seed=55, permute=True, root="random")
    g0, new = _dropped(g, 0.3, seed=6)
    off0 = torch.from_numpy(g0.offsets).cuda()
    col0 = torch.from_numpy(g0.cols).cuda()
    par = rst.build(off0, col0, g.root, "cc_euler")
    init = par.cpu().numpy()
    rst.insert_edges(par, torch.from_numpy(new.astype(np.int32)).cuda(), g.root)
    want, _ = oracle.prrst(g.n, g.offsets, g.cols, g.root, init=init)
    assert np.array_equal(par.cpu().numpy(), want)


def test_insert_rejects_bad_ids_and_cycles():
    import paper_2603_11645_gb300 as rst
    par = torch.tensor([0, 0, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(rst.RstError) as e:
        rst.insert_edges(par, torch.tensor([[0, 9]], dtype=torch.int32, device="cuda"), 0)
    assert e.value.code == 7
    cyc = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(rst.RstError) as e:
        rst.insert_edges(cyc, torch.zeros((0, 2), dtype=torch.int32, device="cuda"), 0)
    assert e.value.code == 4
    # the library stays usable
    ok = torch.tensor([0, 0, 2], dtype=torch.int32, device="cuda")
    rst.insert_edges(ok, torch.tensor([[1, 2]], dtype=torch.int32, device="cuda"), 0)
    assert ok.cpu().tolist() == [0, 0, 1]


@pytest.mark.parametrize("which", ["grid", "rmat", "chain", "er"])
@pytest.mark.parametrize("k", [1, 10, 100, 1000])
def test_insert_small_batches_sparse_and_dense(which, k):
    """Small batches take the sparse rounds (walks to the roots, per-tree path
    reversal); a walk limit of 2 hands over to the dense rounds part-way, a
    limit of 0 uses the dense rounds only; with the canonical flag (the input
    comes from rst_build's canonical form) the final re-rooting touches only
    the merged trees.  Every combination gives the oracle's forest."""
    import paper_2603_11645_gb300 as rst
    g = {"er": lambda: graphs.erdos_renyi(80000, 90000, seed=71),
         "grid": lambda: graphs.grid(400, 300, seed=72, permute=True, root="random"),
         "rmat": lambda: graphs.rmat(16, 8, seed=73, connect=False, offsets_bits=32),
         "chain": lambda: graphs.chain_chords(100000, 0.001, seed=74)}[which]()
    g0, new = _dropped(g, 0.3, seed=7)
    new = new[:k]
    init = oracle.rst(g0.n, g0.offsets, g0.cols, g0.root)
    src0 = np.repeat(np.arange(g0.n), np.diff(g0.offsets)).astype(np.int64)
    keep = src0 < g0.cols
    gk = graphs.from_edges(g.n, np.concatenate([src0[keep], new[:, 0]]),
                           np.concatenate([g0.cols[keep].astype(np.int64), new[:, 1]]), root=g.root)
    root = int(g.root)
    want, _ = oracle.prrst(gk.n, gk.offsets, gk.cols, root, init=init)
    try:
        for limit in (2048, 2, 0):
            rst.set_option("insert_walk_limit", limit)
            for canonical in (False, True):
                got = _gpu_insert(init, new, root, canonical)
                assert np.array_equal(got, want), (limit, canonical)
    finally:
        rst.set_option("insert_walk_limit", 2048)


def test_insert_canonical_flag_matches_the_full_re_rooting():
    """The canonical flag on forests rst_build returned, repeated batches in a
    row (each output is canonical again), against the oracle step by step,
    including a batch that merges the root's tree and one that leaves it alone."""
    import paper_2603_11645_gb300 as rst
    g = graphs.grid(500, 400, seed=81, permute=True, root="random")
    g0, new = _dropped(g, 0.6, seed=9)   # below the bond threshold: many small trees
    off0 = torch.from_numpy(g0.offsets).cuda()
    col0 = torch.from_numpy(g0.cols).cuda()
    par = rst.build(off0, col0, g.root, "cc_euler")
    cur = par.cpu().numpy()
    src0 = np.repeat(np.arange(g0.n), np.diff(g0.offsets)).astype(np.int64)
    keep = src0 < g0.cols
    eu, ev = list(src0[keep]), list(g0.cols[keep].astype(np.int64))
    for lo, hi in ((0, 1), (1, 50), (50, 2000), (2000, 2100)):
        batch = new[lo:hi]
        eu += list(batch[:, 0])
        ev += list(batch[:, 1])
        gk = graphs.from_edges(g.n, eu, ev, root=g.root)
        want, _ = oracle.prrst(gk.n, gk.offsets, gk.cols, g.root, init=cur)
        rst.insert_edges(par, torch.from_numpy(batch.astype(np.int32)).cuda(), g.root, canonical=True)
        got = par.cpu().numpy()
        assert np.array_equal(got, want), (lo, hi)
        cur = got


def test_insert_rejects_unknown_flags():
    import ctypes
    import paper_2603_11645_gb300 as rst
    par = torch.tensor([0, 0, 2], dtype=torch.int32, device="cuda")
    code = rst.lib().rst_insert_edges(3, ctypes.c_void_p(par.data_ptr()), None, 0, 0, 6, None)
    assert code == 1
