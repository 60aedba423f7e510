"""The single-block tail of CC+Euler's contraction rounds (GPU).

Once at most 3,072 components with edges remain, CC+Euler deduplicates the
inter-component list to one entry per component pair and one thread block
finishes the remaining hooking rounds; when the pairs do not fit it hands
back to the grid-wide rounds, which request it again one round later.  The
forest is the same either way (minimum-key hooking gives Kruskal's forest
under the (min, max) keys), so every check here is bit-exact against the
oracle:

* graphs whose contracted pair graph is planar (grids) finish in the tail at
  the first request (no hand-back);
* dense random graphs overflow it: 9,358 distinct pairs among 146
  components (more than the 9,216 the block holds) and 18,510 pairs among
  424 components (more than the 16,384-slot pair table) -- both counts from
  replaying minimum-key hooking on these seeded graphs -- and finish after
  one or more hand-backs;
* the same through the graph-launched rounds (rst_build, rst_cc) and the
  host-stepped rounds (rst_build_noalloc).
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
    L.rst_last_stats.restype = ctypes.c_int
    st = (ctypes.c_longlong * 10)()
    k = L.rst_last_stats(st, 10)
    assert k == 10
    return list(st)


def _cases():
    return [
        ("grid", graphs.grid(300, 200, seed=31, permute=True, root="random"), False),
        ("grid-long", graphs.grid(2000, 40, seed=32, permute=True, root="random"), False),
        ("er-pairs-over-block", graphs.erdos_renyi(40000, 200000, seed=11), True),
        ("er-pairs-over-table", graphs.erdos_renyi(30000, 60000, seed=7), True),
        ("er-many-components", graphs.erdos_renyi(30000, 21000, seed=33), None),
        # four components left after round 1: the grid-wide round finishes
        ("rmat", graphs.rmat(15, 16, seed=34, connect=False, offsets_bits=64), None),
    ]


_CASES = None


def _case(i):
    global _CASES
    if _CASES is None:
        _CASES = _cases()
    return _CASES[i]


@pytest.mark.parametrize("ci", range(6), ids=[c[0] for c in _cases()])
def test_tail_parent_labels_and_tree_set(ci):
    import paper_2603_11645_gb300 as rst
    name, g, backs = _case(ci)
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    st = _stats()
    assert np.array_equal(par, oracle.rst(g.n, g.offsets, g.cols, g.root)), name
    tail_rounds, tail_backs = st[7], st[8]
    if backs is not None:  # these reach few components after round 1's contraction
        assert tail_rounds >= 1, name
        assert (tail_backs >= 1) == backs, name
    assert 1 <= st[0] <= 2 * math.ceil(math.log2(g.n)) + 2 + tail_backs, name
    labels, uv, T = rst.cc(off, col)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert np.array_equal(labels.cpu().numpy(), lab), name
    assert T == len(tu)
    got = uv.cpu().numpy()
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    assert np.array_equal(got[:, 0], tu) and np.array_equal(got[:, 1], tv), name


def _noalloc():
    import paper_2603_11645_gb300 as rst
    f = rst.lib().rst_build_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("ci", [0, 2, 3, 4], ids=["grid", "er-pairs-over-block", "er-pairs-over-table",
                                                  "er-many-components"])
def test_tail_host_stepped_rounds(ci):
    """rst_build_noalloc steps the rounds from the host: the same tail and hand-backs."""
    name, g, backs = _case(ci)
    f = _noalloc()
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    out = torch.full((g.n,), -1, dtype=torch.int32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = f(ctypes.c_void_p(off.data_ptr()), g.offsets_bits, ctypes.c_void_p(col.data_ptr()), g.n, g.A,
             g.root, ctypes.c_void_p(out.data_ptr()), stream)
    assert code == 0
    torch.cuda.synchronize()
    st = _stats()
    assert np.array_equal(out.cpu().numpy(), oracle.rst(g.n, g.offsets, g.cols, g.root)), name
    if backs is not None:
        assert st[7] >= 1
        assert (st[8] >= 1) == backs


def test_tail_repeated_calls_reuse_clean_table():
    """A hand-back leaves the pair table empty: alternate overflowing and fitting graphs."""
    import paper_2603_11645_gb300 as rst
    seq = [_case(3)[1], _case(0)[1], _case(2)[1], _case(1)[1], _case(3)[1]]
    for g in seq:
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
        assert np.array_equal(par, oracle.rst(g.n, g.offsets, g.cols, g.root)), g.name
