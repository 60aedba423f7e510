"""Stage marks of the profiling interface (GPU): every mark by default, only
the named ones under rst_profile_only, and the same parent array either way
(the marks only add events between kernels)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _read(L):
    ms = (ctypes.c_float * 4096)()
    names = (ctypes.c_char_p * 4096)()
    k = L.rst_profile_read(ms, names, 4096)
    return [(names[i].decode(), ms[i]) for i in range(k)]


def test_profile_marks_all_and_filtered():
    import paper_2603_11645_gb300 as rst
    L = rst.lib()
    L.rst_profile_enable.argtypes = [ctypes.c_int]
    L.rst_profile_only.argtypes = [ctypes.c_char_p]
    L.rst_profile_only.restype = None
    L.rst_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    g = graphs.grid(600, 500, seed=51, permute=True, root="random")
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)

    L.rst_profile_only(None)
    L.rst_profile_enable(1)
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    every = _read(L)
    assert np.array_equal(par, want)
    names = [nm for nm, _ in every]
    for nm in ("k_r1_choose", "k_r1_resolve", "k_build_list", "cc_rounds", "k_pairs_succ", "k_lr_walk1"):
        assert nm in names, nm
    assert all(v >= 0.0 for _, v in every)

    L.rst_profile_only(b"k_r1_choose,k_r1_resolve")
    par = rst.build(off, col, g.root, "cc_euler").cpu().numpy()
    some = _read(L)
    L.rst_profile_enable(0)
    L.rst_profile_only(None)
    assert np.array_equal(par, want)
    # two marks recorded: the duration read back belongs to the second, the
    # round-1 resolve kernel alone
    assert [nm for nm, _ in some] == ["k_r1_resolve"]
    assert some[0][1] > 0.0
