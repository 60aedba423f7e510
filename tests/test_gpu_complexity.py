"""Round and level counts of the GPU strategies (Table I's complexity claims).

* CC+Euler: the hooking rounds (round 1 included) stay within
  2 ceil(log2 n) + 2: every round of minimum-key hooking at least halves the
  components that still have edges.
* PR-RST: the GPU runs exactly as many rounds as the oracle's simulation of
  the same rules (the final hook-free round included), also within
  4 ceil(log2 (n + 1)) + 2.
* BFS (every variant): on a connected graph the levels expanded are the
  root's eccentricity + 1 (the last expansion finds nothing), the
  eccentricity taken from the oracle's BFS levels.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stats():
    import paper_2603_11645_gb300 as rst
    L = rst.lib()
    L.rst_last_stats.argtypes = [ctypes.c_void_p, ctypes.c_int]
    st = (ctypes.c_longlong * 8)()
    L.rst_last_stats(st, 8)
    return list(st)


def _cases():
    return [graphs.grid(300, 200, seed=91, permute=True, root="random"),
            graphs.grid(2000, 3, seed=92, permute=True, root="random"),
            graphs.chain_chords(50000, 0.001, seed=93),
            graphs.rmat(15, 16, seed=94, connect=True, offsets_bits=32),
            graphs.random_4regular(20000, seed=95)]


@pytest.mark.parametrize("gi", range(5))
def test_round_and_level_counts(gi):
    import paper_2603_11645_gb300 as rst
    g = _cases()[gi]
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    lg = math.ceil(math.log2(g.n))
    rst.build(off, col, g.root, "cc_euler")
    assert 1 <= _stats()[0] <= 2 * lg + 2, g.name
    rst.build(off, col, g.root, "pr_rst")
    _, want_rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    got_rounds = _stats()[0]
    assert got_rounds == want_rounds, g.name
    assert got_rounds <= 4 * math.ceil(math.log2(g.n + 1)) + 2
    lev, _ = oracle.bfs(g.n, g.offsets, g.cols, g.root)
    assert lev.min() >= 0  # connected
    for strategy in ("bfs", "bfs_device", "bfs_persistent"):
        rst.build(off, col, g.root, strategy)
        assert _stats()[5] == int(lev.max()) + 1, (g.name, strategy)
