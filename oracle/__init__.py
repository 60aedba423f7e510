"""CPU oracle for rooted spanning trees (TEST INFRASTRUCTURE ONLY).

Thin ctypes wrapper over ``rst_oracle.c``.  Only the test suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package; the library itself never does.

Parity status per function (what pins each one, see tests/test_oracle_pins.py):

* ``cc_kruskal``   pinned: brute-force minimum spanning forest on <= 8
                   vertices, closed forms (grid comb), invariants.
* ``root_forest``  pinned: closed forms (path, star), invariants, verifier.
* ``euler_tour``   pinned: closed forms (path, star rooted at centre and at a
                   leaf, hand-derived golden tours), rotation-rule DFS,
                   agreement of its parent with ``root_forest``.
* ``bfs``          pinned: Manhattan levels on grids, brute-force parent rule.
* ``verify``       pinned: Kirchhoff spanning-tree counts (n <= 6), mutations.
* ``prrst``        pinned: its output passes ``verify``; the grafts of its
                   first two rounds follow from the round rules alone; and its
                   edge set and round count equal a derivation of the same
                   rules over whole trees (no parent pointers, no path
                   reversal), also when started from a forest.  From
                   a given forest (edge insertions): hand-derived graft and
                   reversal cases, and the invariants (valid RST of the new
                   graph, every old tree edge kept, only inserted edges added).
* ``bcc``          pinned: brute-force blocks from every simple cycle and cut
                   vertices by deletion (n <= 8), closed forms (cycle, path,
                   star, bowtie, grid), networkx where installed.
* ``tree_depths``  pinned: closed forms (path, star, grid comb), BFS-tree
                   depth equals the BFS level, cycle and range rejection.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

VALID, BAD_ROOT, PARENT_RANGE, NON_EDGE, CYCLE, NOT_SPANNING, COMPONENT_ROOT = range(7)


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"{_SO} missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(_SO)
        P, I64, I32, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.or_cc_kruskal.argtypes = [I64, P, P, P, P, P, P]
        lib.or_root_forest.argtypes = [I64, I64, P, P, I32, P]
        lib.or_euler_tour.argtypes = [I64, I64, P, P, I32, P, P, P, P]
        lib.or_bfs.argtypes = [I64, P, P, I32, P, P]
        lib.or_verify.argtypes = [I64, P, P, I32, P, I]
        if hasattr(lib, "or_prrst"):
            lib.or_prrst.argtypes = [I64, P, P, I32, P, P]
            lib.or_prrst_from.argtypes = [I64, P, P, I32, P, P, P]
        lib.or_bcc.argtypes = [I64, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data


def _csr(offsets, cols):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    col = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return off, col


def cc_kruskal(n, offsets, cols):
    """Return (labels[n], tree_u[T], tree_v[T]) with tree edges u < v in ascending key order."""
    off, col = _csr(offsets, cols)
    lab = np.empty(max(n, 1), dtype=np.int32)
    tu = np.empty(max(n, 1), dtype=np.int32)
    tv = np.empty(max(n, 1), dtype=np.int32)
    t = ctypes.c_int64(0)
    rc = _L().or_cc_kruskal(n, _p(off), _p(col), _p(lab), _p(tu), _p(tv), ctypes.byref(t))
    if rc != 0:
        raise ValueError(f"or_cc_kruskal failed: {rc}")
    T = t.value
    return lab[:n].copy(), tu[:T].copy(), tv[:T].copy()


def root_forest(n, tree_u, tree_v, root):
    tu = np.ascontiguousarray(np.asarray(tree_u, dtype=np.int32))
    tv = np.ascontiguousarray(np.asarray(tree_v, dtype=np.int32))
    T = int(tu.size)
    if T == 0:
        tu = np.zeros(1, np.int32); tv = np.zeros(1, np.int32)
    par = np.empty(max(n, 1), dtype=np.int32)
    rc = _L().or_root_forest(n, T, _p(tu), _p(tv), int(root), _p(par))
    if rc != 0:
        raise ValueError(f"or_root_forest failed: {rc}")
    return par[:n].copy()


def euler_tour(n, tree_u, tree_v, root):
    """Return (src[2T], dst[2T], rank[2T], parent[n]); arcs in sorted (src, dst) order."""
    tu = np.ascontiguousarray(np.asarray(tree_u, dtype=np.int32))
    tv = np.ascontiguousarray(np.asarray(tree_v, dtype=np.int32))
    T = int(tu.size)
    E = 2 * T
    src = np.empty(max(E, 1), np.int32); dst = np.empty(max(E, 1), np.int32)
    rank = np.empty(max(E, 1), np.int32); par = np.empty(max(n, 1), np.int32)
    if T == 0:
        tu = np.zeros(1, np.int32); tv = np.zeros(1, np.int32)
    rc = _L().or_euler_tour(n, T, _p(tu), _p(tv), int(root), _p(src), _p(dst), _p(rank), _p(par))
    if rc != 0:
        raise ValueError(f"or_euler_tour failed: {rc}")
    return src[:E].copy(), dst[:E].copy(), rank[:E].copy(), par[:n].copy()


def bfs(n, offsets, cols, root):
    """Return (level[n], parent[n])."""
    off, col = _csr(offsets, cols)
    lev = np.empty(max(n, 1), np.int32); par = np.empty(max(n, 1), np.int32)
    rc = _L().or_bfs(n, _p(off), _p(col), int(root), _p(lev), _p(par))
    if rc != 0:
        raise ValueError(f"or_bfs failed: {rc}")
    return lev[:n].copy(), par[:n].copy()


def verify(n, offsets, cols, root, parent, strict_roots=True):
    off, col = _csr(offsets, cols)
    par = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    if par.size == 0:
        par = np.zeros(1, np.int32)
    return int(_L().or_verify(n, _p(off), _p(col), int(root), _p(par), 1 if strict_roots else 0))


def rst(n, offsets, cols, root):
    """The reference RST of the CC + Euler pipeline: Kruskal forest rooted at root."""
    lab, tu, tv = cc_kruskal(n, offsets, cols)
    return root_forest(n, tu, tv, root)


def prrst(n, offsets, cols, root, init=None):
    """PR-RST rounds from singletons, or from the rooted forest `init` (the
    incremental case: cols then hold the old edges plus the inserted ones)."""
    off, col = _csr(offsets, cols)
    par = np.empty(max(n, 1), np.int32)
    rounds = ctypes.c_int64(0)
    if init is None:
        rc = _L().or_prrst(n, _p(off), _p(col), int(root), _p(par), ctypes.byref(rounds))
    else:
        ini = np.ascontiguousarray(np.asarray(init, dtype=np.int32))
        rc = _L().or_prrst_from(n, _p(off), _p(col), int(root), _p(ini), _p(par), ctypes.byref(rounds))
    if rc != 0:
        raise ValueError(f"or_prrst failed: {rc}")
    return par[:n].copy(), rounds.value


def tree_depths(n, parent):
    """Depth of every vertex of a rooted forest (edges up to the root; roots
    have parent[v] == v) by walking each parent chain once, remembering the
    depths already known.  Raises ValueError for a parent outside [0, n) or a
    chain that returns to a vertex of its own walk (a cycle).  The tree-shape
    measure of Section IV-B / Fig. 2."""
    par = np.asarray(parent, dtype=np.int64)
    if n and (par.min() < 0 or par.max() >= n):
        raise ValueError("parent out of range")
    depth = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        if depth[v] >= 0:
            continue
        chain = []
        on_chain = set()
        x = v
        while depth[x] < 0 and par[x] != x:
            if x in on_chain:
                raise ValueError("cycle")
            on_chain.add(x)
            chain.append(x)
            x = int(par[x])
        d = 0 if depth[x] < 0 else int(depth[x])  # x is a root or already known
        if depth[x] < 0:
            depth[x] = 0
        for y in reversed(chain):
            d += 1
            depth[y] = d
    return depth


def bcc(n, offsets, cols):
    """Blocks (biconnected components) and cut vertices by Hopcroft-Tarjan
    depth-first search: (label uint32[A], cut uint8[n], number of blocks).
    label[a] is the smallest CSR position among the arcs of arc a's block
    (0xFFFFFFFF for a self-loop)."""
    off, col = _csr(offsets, cols)
    A = int(off[n]) if n > 0 else 0
    label = np.empty(max(A, 1), dtype=np.uint32)
    cut = np.zeros(max(n, 1), dtype=np.uint8)
    nb = ctypes.c_int64(0)
    rc = _L().or_bcc(n, _p(off), _p(col), _p(label), _p(cut), ctypes.byref(nb))
    if rc != 0:
        raise ValueError(f"or_bcc failed: {rc}")
    return label[:A].copy(), cut[:n].copy(), int(nb.value)
