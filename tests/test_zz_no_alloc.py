"""rst_build_noalloc against rst_build and the CPU oracle (GPU).

rst_build_noalloc serves callers that cannot allocate device memory: a serving
process or an embedding runtime that reserves its whole device-memory budget
up front, or a host whose allocator must not be entered from the calling
thread.  It must return exactly the CC+Euler parent array -- the one
rst_build returns and the one the oracle defines -- call after call, although
every call reuses the same fixed workspace inside the library, and the device
memory in use must not change across its calls.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
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
def test_noalloc_equals_rst_build_and_oracle_on_two_calls(gi):
    import paper_2603_11645_gb300 as rst
    g = _cases()[gi]
    f = _entry()
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    col = torch.from_numpy(g.cols).to(dev)
    want = rst.build(off, col, g.root, "cc_euler").clone()
    ref = oracle.rst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(want.cpu().numpy(), ref)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.full((g.n,), -1, dtype=torch.int32, device=dev) for _ in range(3)]

    def call(out):
        return f(ctypes.c_void_p(off.data_ptr()), g.offsets_bits, ctypes.c_void_p(col.data_ptr()),
                 g.n, g.A, g.root, ctypes.c_void_p(out.data_ptr()), stream)

    assert call(outs[0]) == 0  # the first call on the device also does the one-time set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for out in outs[1:]:  # two calls in a row on the shared workspace
        assert call(out) == 0
        torch.cuda.synchronize()
        # integer output: bit-exact, as in every parity test
        assert torch.equal(out, want)
        assert np.array_equal(out.cpu().numpy(), ref)
    assert torch.cuda.mem_get_info(dev)[0] == free0


def test_noalloc_rejects_inputs_beyond_its_limits():
    f = _entry()
    # checked before any GPU work: pointers are never touched
    assert f(None, 32, None, 65537, 10, 0, None, None) == UNSUPPORTED
    assert f(None, 32, None, 100, 524289, 0, None, None) == UNSUPPORTED
