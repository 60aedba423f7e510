"""RST_CC_FAST (sampled union-find connectivity + Euler rooting).

Its tree edges are chosen by races, so parity is checked through what IS
fixed: the oracle verifier's exact verdict (valid rooted spanning forest,
requested root, every other tree rooted at its minimum vertex), the tree-edge
count n - c, the components (labels from the oracle), and the rooting: the
oracle re-roots the returned edge set at the same root and must give back the
same parent array.
"""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    from test_gpu_parity import edge_cases, small_graphs
    return small_graphs() + edge_cases()


def _check(g, par):
    assert oracle.verify(g.n, g.offsets, g.cols, g.root, par) == oracle.VALID, g.name
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    nonroot = par != np.arange(g.n)
    assert int(nonroot.sum()) == len(tu), g.name  # n - c tree edges
    v = np.nonzero(nonroot)[0]
    assert np.array_equal(lab[v], lab[par[v]]), g.name  # edges stay inside components
    again = oracle.root_forest(g.n, v, par[v], g.root)
    assert np.array_equal(again, par), g.name


def test_cc_fast_is_a_valid_rst_on_every_family():
    import paper_2603_11645_gb300 as rst
    for g in _cases():
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        par = rst.build(off, col, g.root, "cc_fast").cpu().numpy()
        _check(g, par)
        assert rst.verify(off, col, g.root, torch.from_numpy(par).cuda()) == 0


def test_cc_fast_repeated_runs_stay_valid():
    import paper_2603_11645_gb300 as rst
    g = graphs.rmat(16, 16, seed=41, connect=False, offsets_bits=32)
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    for _ in range(5):
        _check(g, rst.build(off, col, g.root, "cc_fast").cpu().numpy())


@pytest.mark.parametrize("which", ["grid4096", "rmat20"])
def test_cc_fast_large(which):
    import paper_2603_11645_gb300 as rst
    g = (graphs.workload_grid4096() if which == "grid4096"
         else graphs.rmat(20, 16, seed=42, connect=True, offsets_bits=64))
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = rst.build(off, col, g.root, "cc_fast")
    assert rst.verify(off, col, g.root, par) == 0
    _check(g, par.cpu().numpy())


def test_cc_fast_not_supported_in_batches():
    import paper_2603_11645_gb300 as rst
    b = graphs.pack_batch([graphs.grid(8, 8, seed=1), graphs.grid(5, 9, seed=2)])
    with pytest.raises(rst.RstError) as e:
        rst.build_batch(torch.from_numpy(b.offsets).cuda(), torch.from_numpy(b.cols).cuda(),
                        torch.from_numpy(b.vtx_off).cuda(), torch.from_numpy(b.arc_off).cuda(),
                        torch.from_numpy(b.roots).cuda(), strategy="cc_fast")
    assert e.value.code == 6
