"""Tree depth (rst_tree_depth) against the oracle, on the trees every
strategy returns; the height comparison of CC+Euler and BFS trees."""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    return [graphs.grid(60, 40, seed=31, permute=True, root="random"),
            graphs.grid(1, 300, seed=32, permute=True, root="random"),
            graphs.chain_chords(20000, 0.001, seed=33),
            graphs.rmat(13, 8, seed=34, connect=False, offsets_bits=32),
            graphs.erdos_renyi(3000, 2000, seed=35),
            graphs.from_edges(1, [], [], name="single", root=0),
            graphs.from_edges(5, [], [], name="no-edges", root=2)]


@pytest.mark.parametrize("strategy", ["cc_euler", "bfs", "pr_rst"])
def test_depth_matches_oracle(strategy):
    import paper_2603_11645_gb300 as rst
    for g in _cases():
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        par = rst.build(off, col, g.root, strategy)
        depth, height = rst.tree_depth(par)
        want = oracle.tree_depths(g.n, par.cpu().numpy())
        assert np.array_equal(depth.cpu().numpy(), want), (g.name, strategy)
        assert height == (int(want.max()) if g.n else 0)
        _, h2 = rst.tree_depth(par, want_depths=False)
        assert h2 == height


def test_depth_rejects_cycles_and_bad_parents():
    import paper_2603_11645_gb300 as rst
    cyc = torch.tensor([0, 2, 3, 1, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(rst.RstError) as e:
        rst.tree_depth(cyc)
    assert e.value.code == 4  # iteration bound exceeded: a chain never reaches a root
    bad = torch.tensor([0, 7, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(rst.RstError) as e:
        rst.tree_depth(bad)
    assert e.value.code == 1
    # the library stays usable
    ok = torch.tensor([0, 0, 1], dtype=torch.int32, device="cuda")
    d, h = rst.tree_depth(ok)
    assert d.cpu().tolist() == [0, 1, 2] and h == 2


@pytest.fixture(scope="module")
def grid4096():
    return graphs.workload_grid4096()


def test_grid4096_cc_euler_tree_is_deeper_than_bfs(grid4096):
    """Fig. 2's trade-off on the 4096 x 4096 workload: the BFS tree's height is
    the BFS eccentricity (levels - 1), the CC+Euler tree is deeper; every depth
    satisfies depth[v] = depth[parent[v]] + 1 off the root."""
    import paper_2603_11645_gb300 as rst
    g = grid4096
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    heights = {}
    for s in ("cc_euler", "bfs"):
        par = rst.build(off, col, g.root, s)
        depth, h = rst.tree_depth(par)
        idx = torch.arange(g.n, device="cuda", dtype=torch.int32)
        nonroot = par != idx
        assert int(depth[g.root]) == 0 and int((depth == 0).sum()) == 1
        assert torch.equal(depth[nonroot], depth[par[nonroot].long()] + 1)
        heights[s] = h
    lev, _ = oracle.bfs(g.n, g.offsets, g.cols, g.root)
    assert heights["bfs"] == int(lev.max())
    assert heights["cc_euler"] > heights["bfs"]
