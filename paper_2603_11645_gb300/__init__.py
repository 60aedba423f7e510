"""GB300 rooted-spanning-tree library: Python binding over librst.so.

Argument marshalling only: every step of every strategy runs in the CUDA
kernels of librst.so (include/rst.h).  PyTorch provides device memory and the
current stream.  There is no CPU fallback: if the native library is missing
the first call raises.
"""
from __future__ import annotations

import ctypes
import os

__all__ = ["build", "build_batch", "cc", "euler_root", "verify", "tree_depth", "bcc", "insert_edges", "set_option", "get_option", "lib",
           "RstError", "STRATEGIES"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librst.so")

STRATEGIES = {"auto": 0, "bfs": 1, "cc_euler": 2, "pr_rst": 3, "cc_fast": 4, "bfs_device": 5,
              "bfs_persistent": 6}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "iteration bound exceeded", 5: "timeout", 6: "unsupported", 7: "device-detected error"}

_lib = None


class RstError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


def lib():
    """The loaded librst.so (ctypes.CDLL) with argument types set."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        L.rst_build.argtypes = [P, I, P, I64, I64, I32, I, P, P]
        L.rst_cc.argtypes = [P, I, P, I64, I64, P, P, P, P]
        L.rst_euler_root.argtypes = [I64, P, I64, I32, P, P, P]
        L.rst_verify.argtypes = [P, I, P, I64, I64, I32, P, P, P]
        L.rst_build_batch.argtypes = [P, I, P, P, P, I32, P, I, P, P]
        L.rst_tree_depth.argtypes = [P, I64, P, P, P]
        L.rst_bcc.argtypes = [P, I, P, I64, I64, P, P, P, P]
        L.rst_insert_edges.argtypes = [I64, P, P, I64, I32, ctypes.c_uint, P]
        L.rst_set_option.argtypes = [ctypes.c_char_p, ctypes.c_longlong]
        L.rst_get_option.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong)]
        L.rst_status_string.argtypes = [I]
        L.rst_status_string.restype = ctypes.c_char_p
        L.rst_version.restype = I
        for fn in ("rst_build", "rst_cc", "rst_euler_root", "rst_verify", "rst_shutdown", "rst_set_option", "rst_tree_depth", "rst_bcc", "rst_insert_edges",
                   "rst_get_option"):
            getattr(L, fn).restype = I
        for fn in ("rst_build_batch", "rst_select", "rst_build_batch_graph"):
            if hasattr(L, fn):
                getattr(L, fn).restype = I
        _lib = L
    return _lib


def _check(fn, code):
    if code != 0:
        raise RstError(fn, code)


def set_option(key: str, value: int) -> None:
    """rst_set_option: a tuning knob ("lr_spacing", "round_blocks_per_sm",
    "bfs_bottom_up_divisor") or the BFS level cap ("bfs_max_levels")."""
    _check("rst_set_option", lib().rst_set_option(key.encode(), int(value)))


def get_option(key: str) -> int:
    v = ctypes.c_longlong(0)
    _check("rst_get_option", lib().rst_get_option(key.encode(), ctypes.byref(v)))
    return int(v.value)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _graph_args(offsets, cols):
    import torch
    assert offsets.is_cuda and cols.is_cuda, "offsets and cols must be CUDA tensors"
    assert cols.dtype == torch.int32
    assert offsets.dtype in (torch.int32, torch.int64)
    assert offsets.is_contiguous() and cols.is_contiguous()
    bits = 64 if offsets.dtype == torch.int64 else 32
    n = offsets.numel() - 1
    m = cols.numel()
    return bits, n, m


def build(offsets, cols, root: int, strategy: str = "cc_euler", out=None, stream=None):
    """Rooted spanning tree: returns parent (int32 CUDA tensor of length n)."""
    import torch
    bits, n, m = _graph_args(offsets, cols)
    parent = out if out is not None else torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
    code = lib().rst_build(ctypes.c_void_p(offsets.data_ptr()), bits, ctypes.c_void_p(cols.data_ptr()),
                           n, m, int(root), STRATEGIES[strategy], ctypes.c_void_p(parent.data_ptr()),
                           _stream(stream))
    _check("rst_build", code)
    return parent[:n]


def build_batch(offsets, cols, vtx_off, arc_off, roots, strategy: str = "cc_euler", out=None, stream=None):
    """Rooted spanning trees of a packed batch (layout of include/rst.h):
    returns the packed LOCAL parent array (int32 CUDA tensor)."""
    import torch
    for t in (offsets, cols, vtx_off, arc_off, roots):
        assert t.is_cuda and t.is_contiguous()
    assert vtx_off.dtype == torch.int64 and arc_off.dtype == torch.int64 and roots.dtype == torch.int32
    G = roots.numel()
    N = int(vtx_off[-1].item())
    bits = 64 if offsets.dtype == torch.int64 else 32
    parent = out if out is not None else torch.empty(max(N, 1), dtype=torch.int32, device=offsets.device)
    code = lib().rst_build_batch(ctypes.c_void_p(offsets.data_ptr()), bits, ctypes.c_void_p(cols.data_ptr()),
                                 ctypes.c_void_p(vtx_off.data_ptr()), ctypes.c_void_p(arc_off.data_ptr()), G,
                                 ctypes.c_void_p(roots.data_ptr()), STRATEGIES[strategy],
                                 ctypes.c_void_p(parent.data_ptr()), _stream(stream))
    _check("rst_build_batch", code)
    return parent[:N]


def cc(offsets, cols, stream=None):
    """Connected components: returns (labels[n], tree_uv[T, 2], T)."""
    import torch
    bits, n, m = _graph_args(offsets, cols)
    labels = torch.empty(max(n, 1), dtype=torch.int32, device=offsets.device)
    uv = torch.empty(max(2 * (n - 1), 2), dtype=torch.int32, device=offsets.device)
    t = ctypes.c_int64(0)
    code = lib().rst_cc(ctypes.c_void_p(offsets.data_ptr()), bits, ctypes.c_void_p(cols.data_ptr()), n, m,
                        ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(uv.data_ptr()), ctypes.byref(t),
                        _stream(stream))
    _check("rst_cc", code)
    T = t.value
    return labels[:n], uv[:2 * T].view(T, 2), T


def euler_root(n: int, tree_uv, root: int, with_rank: bool = True, stream=None):
    """Euler-tour rooting of a forest given as a (T, 2) int32 CUDA tensor.

    Returns (parent[n], rank[2T] or None); ranks are indexed by the arcs'
    lexicographic (src, dst) order."""
    import torch
    uv = tree_uv.contiguous().view(-1)
    assert uv.dtype == torch.int32 and uv.is_cuda
    T = uv.numel() // 2
    parent = torch.empty(max(n, 1), dtype=torch.int32, device=uv.device)
    rank = torch.empty(max(2 * T, 1), dtype=torch.int32, device=uv.device) if with_rank else None
    code = lib().rst_euler_root(n, ctypes.c_void_p(uv.data_ptr()), T, int(root), ctypes.c_void_p(parent.data_ptr()),
                                ctypes.c_void_p(rank.data_ptr()) if with_rank else None, _stream(stream))
    _check("rst_euler_root", code)
    return parent[:n], (rank[:2 * T] if with_rank else None)


def verify(offsets, cols, root: int, parent, stream=None) -> int:
    """Exact verdict code of a parent array (0 = valid rooted spanning tree/forest)."""
    bits, n, m = _graph_args(offsets, cols)
    v = ctypes.c_int32(-1)
    code = lib().rst_verify(ctypes.c_void_p(offsets.data_ptr()), bits, ctypes.c_void_p(cols.data_ptr()), n, m,
                            int(root), ctypes.c_void_p(parent.data_ptr()), ctypes.byref(v), _stream(stream))
    _check("rst_verify", code)
    return int(v.value)


def tree_depth(parent, want_depths: bool = True, stream=None):
    """Depth of every vertex of a rooted forest (device int32 tensor, or None)
    and the forest's height."""
    import torch
    assert parent.is_cuda and parent.dtype == torch.int32 and parent.is_contiguous()
    n = parent.numel()
    depth = torch.empty(n, dtype=torch.int32, device=parent.device) if want_depths else None
    mx = ctypes.c_int64(0)
    code = lib().rst_tree_depth(ctypes.c_void_p(parent.data_ptr()), n,
                                ctypes.c_void_p(depth.data_ptr()) if depth is not None else None,
                                ctypes.byref(mx), _stream(stream))
    _check("rst_tree_depth", code)
    return depth, int(mx.value)


def bcc(offsets, cols, want_cut: bool = True, stream=None):
    """Blocks and cut vertices: (block label per arc as an int32 tensor holding
    the uint32 values, -1 for self-loops; cut flags uint8 tensor or None;
    number of blocks)."""
    import torch
    bits, n, m = _graph_args(offsets, cols)
    label = torch.empty(m, dtype=torch.int32, device=cols.device)
    cut = torch.empty(n, dtype=torch.uint8, device=cols.device) if want_cut else None
    nb = ctypes.c_int64(0)
    code = lib().rst_bcc(ctypes.c_void_p(offsets.data_ptr()), bits, ctypes.c_void_p(cols.data_ptr()), n, m,
                         ctypes.c_void_p(label.data_ptr()) if m else None,
                         ctypes.c_void_p(cut.data_ptr()) if cut is not None else None,
                         ctypes.byref(nb), _stream(stream))
    _check("rst_bcc", code)
    return label, cut, int(nb.value)


def insert_edges(parent, new_uv, root: int, canonical: bool = False, stream=None):
    """Updates the rooted spanning forest `parent` (int32 CUDA tensor, in
    place) after inserting the undirected edges of `new_uv` (int32 CUDA
    tensor of shape (k, 2)); returns `parent`.  canonical=True declares that
    `parent` is in the canonical form rst_build returns for `root`
    (RST_INSERT_CANONICAL)."""
    import torch
    assert parent.is_cuda and parent.dtype == torch.int32 and parent.is_contiguous()
    uv = new_uv.contiguous()
    assert uv.is_cuda and uv.dtype == torch.int32 and (uv.numel() == 0 or uv.shape[-1] == 2)
    k = uv.numel() // 2
    code = lib().rst_insert_edges(parent.numel(), ctypes.c_void_p(parent.data_ptr()),
                                  ctypes.c_void_p(uv.data_ptr()) if k else None, k, int(root),
                                  1 if canonical else 0, _stream(stream))
    _check("rst_insert_edges", code)
    return parent
