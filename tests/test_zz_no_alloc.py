"""rst_build_noalloc against rst_build (GPU).

rst_build_noalloc serves callers that cannot allocate memory -- code running
inside a CUDA stream capture, where cudaMalloc is not permitted, or hosts with
a device-memory budget fixed in advance.  It must return exactly the parent
array rst_build returns with the CC+Euler strategy, call after call, even
though every call reuses the same fixed workspace inside the library.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UNSUPPORTED = 6


def _entry():
    import paper_2603_11645_gb300 as rst
    f = rst.lib().rst_build_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _cases():
    return [graphs.workload_grid256(),
            graphs.rmat(12, 8, seed=21, connect=False, offsets_bits=64),
            graphs.erdos_renyi(5000, 9000, seed=3),
            # at the documented limits: 65,536 vertices, just under 524,288 arcs
            graphs.erdos_renyi(65536, 262000, seed=5)]


@pytest.mark.parametrize("gi", range(4))
def test_noalloc_equals_rst_build_on_two_calls(gi):
    import paper_2603_11645_gb300 as rst
    g = _cases()[gi]
    f = _entry()
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    want = rst.build(off, col, g.root, "cc_euler").clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((g.n,), -1, dtype=torch.int32, device=dev)
        code = f(ctypes.c_void_p(off.data_ptr()), g.offsets_bits, ctypes.c_void_p(col.data_ptr()),
                 g.n, g.A, g.root, ctypes.c_void_p(out.data_ptr()), stream)
        assert code == 0
        torch.cuda.synchronize()
        assert torch.equal(out, want)  # integer output: bit-exact, as in every parity test


def test_noalloc_rejects_inputs_beyond_its_limits():
    f = _entry()
    # checked before any GPU work: pointers are never touched
    assert f(None, 32, None, 65537, 10, 0, None, None) == UNSUPPORTED
    assert f(None, 32, None, 100, 524289, 0, None, None) == UNSUPPORTED
