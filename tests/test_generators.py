"""The synthetic input generators (CPU): every graph meets the library's CSR
contract (symmetric, rows sorted ascending, no self-loops, no duplicate arcs,
ids in range), the families have the shapes the workload recipe states, and
everything is reproducible from its seed."""
import numpy as np
import pytest

from paper_2603_11645_gb300 import graphs


def check_contract(g):
    off = g.offsets.astype(np.int64)
    col = g.cols.astype(np.int64)
    assert off.shape == (g.n + 1,) and off[0] == 0 and off[-1] == len(col) == g.A
    assert np.all(np.diff(off) >= 0)
    if len(col) == 0:
        return
    assert col.min() >= 0 and col.max() < g.n
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(off))
    same_row = src[1:] == src[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row]), "rows sorted, no duplicate arcs"
    assert not np.any(src == col), "no self-loops"
    fwd = np.sort(src * g.n + col)
    rev = np.sort(col * g.n + src)
    assert np.array_equal(fwd, rev), "symmetric"


def components(g):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    a = csr_matrix((np.ones(g.A), g.cols, g.offsets.astype(np.int64)), shape=(g.n, g.n))
    return connected_components(a, directed=False)[0]


def test_permutation_is_a_seeded_bijection():
    for n in (1, 2, 17, 1000):
        p = graphs.permutation(n, 5)
        assert np.array_equal(np.sort(p), np.arange(n))
        assert np.array_equal(p, graphs.permutation(n, 5))
    assert not np.array_equal(graphs.permutation(1000, 5), graphs.permutation(1000, 6))


def test_uniform_is_in_range_reproducible_and_flat():
    x = graphs.uniform(200_000, 10, 9)
    assert x.min() >= 0 and x.max() < 10
    assert np.array_equal(x, graphs.uniform(200_000, 10, 9))
    counts = np.bincount(x, minlength=10)
    assert np.all(np.abs(counts - 20_000) < 1_000)   # ~7 standard deviations


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (5, 4), (64, 48)])
@pytest.mark.parametrize("permute", [False, True])
def test_grid_shape(W, H, permute):
    g = graphs.grid(W, H, seed=3, permute=permute, root="corner")
    check_contract(g)
    assert g.n == W * H and g.m == H * (W - 1) + W * (H - 1)
    deg = np.diff(g.offsets.astype(np.int64))
    ref = np.diff(graphs.grid(W, H, permute=False).offsets.astype(np.int64))
    assert np.array_equal(np.sort(deg), np.sort(ref))   # relabelling keeps the degrees
    if W >= 2 and H >= 2:
        assert (deg == 4).sum() == (W - 2) * (H - 2) and (deg == 2).sum() == 4
    assert components(g) == 1
    pi = graphs.permutation(W * H, 3) if permute else np.arange(W * H)
    assert g.root == int(pi[0])
    # vertex (i, j) = i*W + j is adjacent to (i, j+1) and (i+1, j) after relabelling
    row = lambda x: g.cols[g.offsets[x]:g.offsets[x + 1]]
    if W >= 2:
        assert int(pi[1]) in row(int(pi[0]))
    if H >= 2:
        assert int(pi[W]) in row(int(pi[0]))


def test_grid_root_modes_and_seeds():
    a = graphs.grid(30, 20, seed=1, root="random")
    b = graphs.grid(30, 20, seed=1, root="random")
    c = graphs.grid(30, 20, seed=2, root="random")
    assert a.root == b.root and np.array_equal(a.cols, b.cols)
    assert not np.array_equal(a.cols, c.cols)
    assert graphs.grid(30, 20, root=17).root == 17


def test_chain_chords_contains_its_path():
    g = graphs.chain_chords(3000, 0.01, seed=4, permute=False)
    check_contract(g)
    for i in (0, 1, 1500, 2998):
        assert i + 1 in g.cols[g.offsets[i]:g.offsets[i + 1]]
    assert (g.n - 1) <= g.m <= (g.n - 1) + 30
    assert components(g) == 1
    p = graphs.chain_chords(3000, 0.01, seed=4, permute=True)
    check_contract(p)
    assert p.m == g.m


def test_rmat_is_skewed_simple_and_connected():
    g = graphs.rmat(12, 8, seed=5, connect=True)
    check_contract(g)
    assert g.offsets.dtype == np.int64 and g.root == 0 and g.n == 4096
    assert components(g) == 1
    deg = np.diff(g.offsets)
    assert deg.max() > 10 * deg.mean()           # heavy-tailed degrees
    h = graphs.rmat(12, 8, seed=5, connect=False, offsets_bits=32)
    check_contract(h)
    assert h.offsets.dtype == np.int32
    assert g.m - h.m == g.meta["connect_edges"]  # one edge per other component
    assert np.array_equal(g.cols, graphs.rmat(12, 8, seed=5, connect=True).cols)


def test_random_4regular_and_erdos_renyi():
    g = graphs.random_4regular(1001, seed=6)
    check_contract(g)
    assert np.all(np.diff(g.offsets) == 4)
    e = graphs.erdos_renyi(5000, 12000, seed=7)
    check_contract(e)
    assert 0 < e.m <= 12000 and 0 <= e.root < 5000


def test_named_workload_sizes():
    g = graphs.workload_grid256()
    assert (g.n, g.m) == (65_536, 130_560)
    assert g.root == int(graphs.permutation(65_536, 1)[0])
    # the 4096 x 4096 headline: the stated counts follow from the grid formula
    assert 4096 * 4096 == 16_777_216 and 2 * 4096 * 4095 == 33_546_240


def test_pack_batch_layout():
    members = [graphs.grid(5, 4, seed=1), graphs.chain_chords(50, 0.1, seed=2),
               graphs.from_edges(3, [], [], root=2), graphs.rmat(6, 4, seed=3, offsets_bits=32)]
    b = graphs.pack_batch(members)
    assert list(b.vtx_off) == list(np.cumsum([0] + [g.n for g in members]))
    assert list(b.arc_off) == list(np.cumsum([0] + [g.A for g in members]))
    for i, g in enumerate(members):
        o = b.offsets[b.vtx_off[i] + i: b.vtx_off[i + 1] + i + 1]
        assert np.array_equal(o, g.offsets.astype(o.dtype))      # local offsets
        assert np.array_equal(b.cols[b.arc_off[i]:b.arc_off[i + 1]], g.cols)
        assert b.roots[i] == g.root


def test_batch_families_and_sizes():
    s = graphs.batch_sizes(500, 1024, 4096, seed=4)
    assert s.min() >= 1024 and s.max() <= 4096
    assert np.array_equal(s, graphs.batch_sizes(500, 1024, 4096, seed=4))
    b = graphs.workload_batch(G=12, lo=1024, hi=2048, seed=4)
    fams = [g.meta.get("family") for g in b.graphs]
    assert fams[:3] == ["grid", "chain", "rmat"] and fams[3:6] == fams[:3]
    for g in b.graphs:
        check_contract(g)
