"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact comparisons (integer work): parent arrays of CC+Euler and BFS,
component labels, the tree edge SET (the list order is unspecified), Euler
ranks indexed by lexicographic arc order, and verifier verdict codes.
"""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(g):
    d = torch.device("cuda:0")
    return torch.from_numpy(g.offsets).to(d), torch.from_numpy(g.cols).to(d)


def small_graphs():
    out = []
    for (W, H, seed) in [(16, 16, 1), (33, 7, 2), (1, 50, 3), (50, 1, 4), (129, 65, 5)]:
        out.append(graphs.grid(W, H, seed=seed, permute=True, root="random"))
    out.append(graphs.grid(40, 30, permute=False, root=0))
    for n, d, s in [(2000, 0.0, 1), (5000, 0.001, 2), (3000, 0.05, 3), (777, 0.5, 4)]:
        out.append(graphs.chain_chords(n, d, seed=s))
    out.append(graphs.erdos_renyi(3000, 2000, seed=7))
    out.append(graphs.erdos_renyi(5000, 12000, seed=8))
    out.append(graphs.rmat(12, 8, seed=9, connect=False, offsets_bits=64))
    out.append(graphs.rmat(14, 16, seed=10, connect=True, offsets_bits=64))
    out.append(graphs.rmat(11, 16, seed=11, connect=True, offsets_bits=32))
    out.append(graphs.random_4regular(4001, seed=12))
    return out


SMALL = None
N_SMALL = 16


def _small():
    global SMALL
    if SMALL is None:
        SMALL = small_graphs()
    return SMALL


def edge_cases():
    cases = []
    cases.append(graphs.from_edges(1, [], [], name="single", root=0))
    cases.append(graphs.from_edges(2, [0], [1], name="one-edge", root=1))
    cases.append(graphs.from_edges(5, [], [], name="no-edges", root=3))
    cases.append(graphs.from_edges(6, [0, 1, 3], [1, 2, 4], name="root-isolated", root=5))
    cases.append(graphs.from_edges(7, [0, 2, 4, 5], [1, 3, 5, 6], name="root-small-comp", root=3))
    cases.append(graphs.from_edges(6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], name="path-root-mid", root=2))
    g = graphs.from_edges(5, [0, 0, 0, 0], [1, 2, 3, 4], name="star64", root=4, offsets_bits=64)
    cases.append(g)
    cases.append(graphs.from_edges(9, [0] * 8, list(range(1, 9)), name="star-centre-root", root=0))
    cases.append(graphs.from_edges(9, [0] * 8, list(range(1, 9)), name="star-leaf-root", root=5))
    cases.append(graphs.from_edges(2, [0], [1], name="pair-root0", root=0))
    cases.append(graphs.from_edges(8, [0, 1, 2, 4, 5, 6], [1, 2, 3, 5, 6, 7], name="two-paths", root=3))
    return cases


def _ids(gs):
    return [g.name for g in gs]


@pytest.mark.parametrize("gi", range(N_SMALL))
def test_cc_euler_parent_small(gi):
    g = _small()[gi]
    off, col = dev(g)
    import paper_2603_11645_gb300 as rst
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(par, want), g.name


@pytest.mark.parametrize("g", edge_cases(), ids=_ids(edge_cases()))
def test_cc_euler_edge_cases(g):
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    assert np.array_equal(par, oracle.rst(g.n, g.offsets, g.cols, g.root))
    labels, uv, T = rst.cc(off, col)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert np.array_equal(labels.cpu().numpy(), lab)
    assert T == len(tu)


@pytest.mark.parametrize("gi", range(N_SMALL))
def test_cc_labels_and_tree_set(gi):
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    labels, uv, T = rst.cc(off, col)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert np.array_equal(labels.cpu().numpy(), lab)
    assert T == len(tu)
    got = uv.cpu().numpy()
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    assert np.array_equal(got[:, 0], tu) and np.array_equal(got[:, 1], tv)


@pytest.mark.parametrize("gi", range(N_SMALL))
def test_euler_root_ranks(gi):
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    # feed the tree edges in a scrambled order and orientation
    rng = np.random.default_rng(gi)
    perm = rng.permutation(len(tu))
    flip = rng.random(len(tu)) < 0.5
    a = np.where(flip, tv, tu)[perm]
    b = np.where(flip, tu, tv)[perm]
    uv = torch.from_numpy(np.stack([a, b], 1).astype(np.int32)).cuda()
    par, rank = rst.euler_root(g.n, uv, g.root)
    s, d, r, p = oracle.euler_tour(g.n, tu, tv, g.root)
    assert np.array_equal(par.cpu().numpy(), p)
    assert np.array_equal(rank.cpu().numpy(), r)


@pytest.mark.parametrize("gi", range(N_SMALL))
def test_bfs_parent_small(gi):
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, "bfs").cpu().numpy()
    lev, want = oracle.bfs(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(par, want), g.name


@pytest.mark.parametrize("g", edge_cases(), ids=_ids(edge_cases()))
def test_bfs_edge_cases(g):
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, "bfs").cpu().numpy()
    assert np.array_equal(par, oracle.bfs(g.n, g.offsets, g.cols, g.root)[1])


DEVICE_BFS = ("bfs_device", "bfs_persistent")


@pytest.mark.parametrize("strategy", DEVICE_BFS)
@pytest.mark.parametrize("gi", range(N_SMALL))
def test_bfs_device_parent_small(gi, strategy):
    """The device-driven level loops (graph while node; persistent kernel)
    give the oracle's BFS tree."""
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, strategy).cpu().numpy()
    assert np.array_equal(par, oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]), g.name


@pytest.mark.parametrize("strategy", DEVICE_BFS)
@pytest.mark.parametrize("g", edge_cases(), ids=_ids(edge_cases()))
def test_bfs_device_edge_cases(g, strategy):
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, strategy).cpu().numpy()
    assert np.array_equal(par, oracle.bfs(g.n, g.offsets, g.cols, g.root)[1])


@pytest.mark.parametrize("strategy", DEVICE_BFS)
def test_bfs_device_long_rows_and_many_components(strategy):
    """Rows longer than one block and than the long-row threshold (a star
    centre with 300,000 leaves, a hub of 5,000), both search directions, and
    components found by the device-side seek far apart in id order."""
    import paper_2603_11645_gb300 as rst
    n = 400_000
    u = [0] * 300_000 + [300_001] * 5_000 + list(range(350_000, 399_999))
    v = list(range(1, 300_001)) + list(range(300_002, 305_002)) + list(range(350_001, 400_000))
    # a few isolated vertices and two-vertex components in the gaps
    u += [310_000, 320_000, 340_000]
    v += [310_001, 320_002, 345_000]
    for root in (0, 300_001, 350_500, 310_000, 305_500):
        g = graphs.from_edges(n, u, v, name="hubs", root=root)
        off, col = dev(g)
        want = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
        for div in (20, 1, 10**6):  # default, always top-down, always bottom-up
            if root == 350_500 and div == 10**6:
                # forced bottom-up steps over the 50,000-level path while the
                # star centre (a 300,000-arc row in another component) is
                # unvisited: every level rescans that row (~30 ms a level)
                continue
            rst.set_option("bfs_bottom_up_divisor", div)
            try:
                par = rst.build(off, col, g.root, strategy).cpu().numpy()
            finally:
                rst.set_option("bfs_bottom_up_divisor", 20)
            assert np.array_equal(par, want), (root, div)


@pytest.mark.parametrize("strategy", DEVICE_BFS)
def test_bfs_device_level_cap(strategy):
    """The level cap ends the device loop with an error status, and the next
    call without a cap is exact again."""
    import paper_2603_11645_gb300 as rst
    g = graphs.chain_chords(5000, 0.0, seed=3)
    off, col = dev(g)
    rst.set_option("bfs_max_levels", 100)
    try:
        with pytest.raises(rst.RstError) as e:
            rst.build(off, col, g.root, strategy)
        assert e.value.code == 4
    finally:
        rst.set_option("bfs_max_levels", 0)
    par = rst.build(off, col, g.root, strategy).cpu().numpy()
    assert np.array_equal(par, oracle.bfs(g.n, g.offsets, g.cols, g.root)[1])


@pytest.mark.parametrize("gi", [0, 3, 6, 8, 10, 12, 15])
def test_verify_matches_oracle(gi):
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = oracle.rst(g.n, g.offsets, g.cols, g.root)
    rng = np.random.default_rng(gi)
    variants = [par.copy()]
    nonroot = np.flatnonzero(par != np.arange(g.n))
    for k in range(12):
        p = par.copy()
        v = int(rng.choice(nonroot)) if len(nonroot) else 0
        kind = k % 6
        if kind == 0:
            p[g.root] = (g.root + 1) % g.n
        elif kind == 1:
            p[v] = g.n + 5
        elif kind == 2:
            p[v] = int(rng.integers(0, g.n))
        elif kind == 3 and p[v] != g.root:
            p[p[v]] = v
        elif kind == 4:
            p[v] = v
        elif kind == 5:
            p = rng.integers(0, g.n, g.n).astype(np.int32)
        variants.append(p)
    for p in variants:
        want = oracle.verify(g.n, g.offsets, g.cols, g.root, p)
        got = rst.verify(off, col, g.root, torch.from_numpy(p.astype(np.int32)).cuda())
        assert got == want


# ------------------------------------------------------------------ named workloads

@pytest.fixture(scope="module")
def grid256():
    return graphs.workload_grid256()


def test_grid256_all_outputs(grid256):
    g = grid256
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(rst.build(off, col, g.root, "cc_euler").cpu().numpy(), want)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    uv = torch.from_numpy(np.stack([tu, tv], 1).astype(np.int32)).cuda()
    par, rank = rst.euler_root(g.n, uv, g.root)
    s, d, r, p = oracle.euler_tour(g.n, tu, tv, g.root)
    assert np.array_equal(rank.cpu().numpy(), r)
    wb = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
    assert np.array_equal(rst.build(off, col, g.root, "bfs").cpu().numpy(), wb)
    for strategy in DEVICE_BFS:
        assert np.array_equal(rst.build(off, col, g.root, strategy).cpu().numpy(), wb), strategy
    assert rst.verify(off, col, g.root, torch.from_numpy(want).cuda()) == 0
    pr = rst.build(off, col, g.root, "pr_rst")
    assert np.array_equal(pr.cpu().numpy(), oracle.prrst(g.n, g.offsets, g.cols, g.root)[0])
    assert rst.verify(off, col, g.root, pr) == 0


@pytest.fixture(scope="module")
def grid4096():
    return graphs.workload_grid4096()


def test_grid4096_cc_euler_and_bfs(grid4096):
    """Full-size high-diameter workload in the configuration the benchmark times."""
    g = grid4096
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)
    got = rst.build(off, col, g.root, "cc_euler")
    assert np.array_equal(got.cpu().numpy(), want)
    assert rst.verify(off, col, g.root, got) == 0
    wb = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
    bpar = rst.build(off, col, g.root, "bfs").cpu().numpy()
    assert np.array_equal(bpar, wb)
    for strategy in DEVICE_BFS:
        assert np.array_equal(rst.build(off, col, g.root, strategy).cpu().numpy(), wb), strategy


@pytest.mark.slow
def test_grid4096_prrst(grid4096):
    """PR-RST on the full-size high-diameter workload (the graph and launch
    configuration the benchmark times), bit-exact against the oracle's
    round-by-round simulation, and a valid RST."""
    g = grid4096
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    got = rst.build(off, col, g.root, "pr_rst")
    want, rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(got.cpu().numpy(), want)
    assert rst.verify(off, col, g.root, got) == 0


@pytest.fixture(scope="module")
def rmat24():
    return graphs.workload_rmat24()


@pytest.mark.slow
def test_rmat24_cc_euler(rmat24):
    g = rmat24
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)
    got = rst.build(off, col, g.root, "cc_euler")
    assert np.array_equal(got.cpu().numpy(), want)
    wb = oracle.bfs(g.n, g.offsets, g.cols, g.root)[1]
    bpar = rst.build(off, col, g.root, "bfs").cpu().numpy()
    assert np.array_equal(bpar, wb)
    for strategy in DEVICE_BFS:
        assert np.array_equal(rst.build(off, col, g.root, strategy).cpu().numpy(), wb), strategy


@pytest.mark.slow
def test_rmat24_prrst(rmat24):
    """PR-RST on the power-law workload (int64 offsets, a hub of ~8M extra
    arcs), bit-exact against the oracle, and a valid RST."""
    g = rmat24
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    got = rst.build(off, col, g.root, "pr_rst")
    want, rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(got.cpu().numpy(), want)
    assert rst.verify(off, col, g.root, got) == 0


# ------------------------------------------------------------------ PR-RST

@pytest.mark.parametrize("gi", range(N_SMALL))
def test_prrst_matches_oracle(gi):
    """Bit-exact against the oracle's round-by-round simulation of the same
    hooking rule, and a valid RST."""
    g = _small()[gi]
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, "pr_rst")
    want, rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(par.cpu().numpy(), want), g.name
    assert rst.verify(off, col, g.root, par) == 0


@pytest.mark.parametrize("g", edge_cases(), ids=_ids(edge_cases()))
def test_prrst_edge_cases(g):
    import paper_2603_11645_gb300 as rst
    off, col = dev(g)
    par = rst.build(off, col, g.root, "pr_rst").cpu().numpy()
    assert np.array_equal(par, oracle.prrst(g.n, g.offsets, g.cols, g.root)[0])


def test_list_ranking_head_on_a_splitter_after_other_calls():
    """A path rooted at 0 puts the tour head at sorted position 0 (a regular
    splitter of the list ranking) with enough arcs for several levels; run it
    after calls that leave other data in the shared workspace."""
    import paper_2603_11645_gb300 as rst
    n = 100_000
    g = graphs.from_edges(n, list(range(n - 1)), list(range(1, n)), root=0)
    other = graphs.erdos_renyi(150_000, 300_000, seed=77)
    oo, oc = dev(other)
    rst.build(oo, oc, other.root, "bfs")
    rst.build(oo, oc, other.root, "cc_euler")
    off, col = dev(g)
    par = rst.build(off, col, 0, "cc_euler").cpu().numpy()
    assert par[0] == 0 and np.array_equal(par[1:], np.arange(n - 1))
    uv = torch.from_numpy(np.stack([np.arange(n - 1), np.arange(1, n)], 1).astype(np.int32)).cuda()
    p2, rank = rst.euler_root(n, uv, 0)
    r = rank.cpu().numpy()
    # sorted arcs: (0,1), then per vertex i >= 1: (i,i-1), (i,i+1)
    assert r[0] == 0 and np.array_equal(p2.cpu().numpy(), par)


def test_euler_root_rejects_non_forests_then_recovers():
    """An edge list with a cycle or a repeated edge is not a forest: the call
    fails with an error code (its connectivity pass finds fewer tree edges
    than given), and the next call on a forest is exact again, with and
    without ranks (the two list-ranking exits)."""
    import paper_2603_11645_gb300 as rst
    n = 9
    bad = [
        ([0, 1, 2, 3, 5, 6], [1, 2, 3, 0, 6, 7]),   # a 4-cycle next to a path
        ([0, 1, 1, 4], [1, 2, 2, 5]),               # a repeated edge
    ]
    for u, v in bad:
        uv = torch.tensor(np.stack([u, v], 1), dtype=torch.int32, device="cuda")
        for with_rank in (False, True):
            with pytest.raises(rst.RstError):
                rst.euler_root(n, uv, 0, with_rank=with_rank)
    g = graphs.grid(300, 200, seed=21, permute=True, root="random")
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    uv = torch.from_numpy(np.stack([tu, tv], 1).astype(np.int32)).cuda()
    s, d, r, p = oracle.euler_tour(g.n, tu, tv, g.root)
    par, rank = rst.euler_root(g.n, uv, g.root)
    assert np.array_equal(par.cpu().numpy(), p) and np.array_equal(rank.cpu().numpy(), r)
    par2, _ = rst.euler_root(g.n, uv, g.root, with_rank=False)
    assert np.array_equal(par2.cpu().numpy(), p)
