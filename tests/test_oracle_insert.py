"""Pins of the PR-RST oracle started from an existing rooted forest (edge
insertions): hand-derived graft/reversal cases and the invariants any correct
insertion must keep."""
import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs


def _graph(n, edges):
    return graphs.from_edges(n, [e[0] for e in edges], [e[1] for e in edges], root=0)


@pytest.mark.parametrize("n,old,init,new,root,want", [
    # path 0-1-2 rooted at 0 and the singleton 3; (2,3): tree {3} hooks under 2
    (4, [(0, 1), (1, 2)], [0, 0, 1, 3], [(2, 3)], 0, [0, 0, 1, 2]),
    # path 0-1-2 and tree 3-4 rooted at 3; (4,1): the minimum rule lets tree 3
    # hook; it is re-rooted at 4 (3 now under 4) and 4 grafts under 1
    (5, [(0, 1), (1, 2), (3, 4)], [0, 0, 1, 3, 3], [(4, 1)], 0, [0, 0, 1, 4, 1]),
    # the same with root 4: the final re-rooting reverses 4 -> 1 -> 0
    (5, [(0, 1), (1, 2), (3, 4)], [0, 0, 1, 3, 3], [(4, 1)], 4, [1, 4, 1, 4, 4]),
    # trees {0,5} (root 0) and {1,6} (root 1) joined by (5,6) and (0,1): tree 1
    # takes its smallest eligible arc, 1->0; the singletons 2,3,4 stay roots
    (7, [(0, 5), (1, 6)], [0, 0, 2, 3, 4, 0, 1], [(5, 6), (0, 1)], 0, [0, 0, 2, 3, 4, 0, 1]),
])
def test_insert_hand_derived(n, old, init, new, root, want):
    g = _graph(n, old + new)
    got, _ = oracle.prrst(n, g.offsets, g.cols, root, init=init)
    assert got.tolist() == want


def test_insert_from_singletons_is_plain_prrst():
    g = graphs.erdos_renyi(500, 700, seed=3)
    a, ra = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    b, rb = oracle.prrst(g.n, g.offsets, g.cols, g.root, init=np.arange(g.n))
    assert np.array_equal(a, b) and ra == rb


def test_insert_rejects_a_cyclic_forest():
    g = _graph(3, [(0, 1), (1, 2)])
    with pytest.raises(ValueError):
        oracle.prrst(3, g.offsets, g.cols, 0, init=[1, 2, 0])


def _edges_of(par):
    v = np.nonzero(par != np.arange(len(par)))[0]
    return {(int(min(a, b)), int(max(a, b))) for a, b in zip(v, par[v])}


@pytest.mark.parametrize("seed", range(8))
def test_insert_invariants(seed):
    rng = np.random.default_rng(seed)
    n = 400
    g0 = graphs.erdos_renyi(n, int(rng.integers(150, 500)), seed=seed)
    forest = oracle.rst(n, g0.offsets, g0.cols, g0.root)
    src = np.repeat(np.arange(n), np.diff(g0.offsets))
    old = [(int(a), int(b)) for a, b in zip(src, g0.cols) if a < b]
    new = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(int(rng.integers(1, 200)))]
    new = [(min(a, b), max(a, b)) for a, b in new if a != b]
    allE = sorted(set(old) | set(new))
    g1 = _graph(n, allE)
    root = int(rng.integers(0, n))
    res, _ = oracle.prrst(n, g1.offsets, g1.cols, root, init=forest)
    assert oracle.verify(n, g1.offsets, g1.cols, root, res) == oracle.VALID
    before, after = _edges_of(forest), _edges_of(res)
    assert before <= after                          # every old tree edge kept
    assert after - before <= set(new)               # only inserted edges added
    lab, tu, tv = oracle.cc_kruskal(n, g1.offsets, g1.cols)
    assert len(after) == len(tu)                    # n - c tree edges
