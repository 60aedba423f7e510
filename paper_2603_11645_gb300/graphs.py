"""Seeded synthetic graph generators (inputs only, no spanning-tree arithmetic).

The paper evaluates on SNAP/SuiteSparse graphs (Section IV, Table II) that
split into two shapes: high-diameter, low-degree road/OSM meshes and
low-diameter power-law web/social/Kronecker graphs. These generators make
seeded stand-ins of both shapes:

* ``grid``          W x H 4-neighbour mesh, vertex ids permuted (road-like)
* ``chain_chords``  a path with uniformly random chords (diameter knob)
* ``rmat``          R-MAT power-law graph, symmetrised, deduplicated and made
                    connected by one edge from each other component's minimum
                    vertex to vertex 0 (Kronecker-like)
* ``random_4regular`` union of two random Hamiltonian cycles

Every generator returns a :class:`Graph` whose CSR is symmetric, has sorted
rows, no self-loops and no duplicate arcs: the input contract of the library.
The heavy lifting (RNG, R-MAT draws, CSR packing) is in ``gen/graphgen.c``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SO = os.path.join(_HERE, "gen", "libgraphgen.so")
_lib = None


def _gen():
    global _lib
    if _lib is None:
        if not os.path.exists(_GEN_SO):
            raise RuntimeError(
                f"{_GEN_SO} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(_GEN_SO)
        P = ctypes.c_void_p
        I64, U64, I32, D = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        lib.gg_permutation.argtypes = [I64, U64, P]
        lib.gg_uniform.argtypes = [I64, U64, U64, P]
        lib.gg_rmat_edges.argtypes = [ctypes.c_int, I64, D, D, D, U64, P, P]
        lib.gg_build_csr.argtypes = [I64, I64, P, P, P, P]
        lib.gg_build_csr.restype = I64
        lib.gg_connect_to_zero.argtypes = [I64, I64, P, P, P, P]
        lib.gg_connect_to_zero.restype = I64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class Graph:
    """Symmetric CSR graph with sorted rows (int32 ids)."""

    name: str
    n: int
    offsets: np.ndarray          # int32 or int64, length n+1
    cols: np.ndarray             # int32, length A = offsets[n]
    root: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def A(self) -> int:
        """Number of stored directed arcs (CSR nnz)."""
        return int(self.offsets[self.n])

    @property
    def m(self) -> int:
        """Number of undirected edges (the unit of the edges/s metric)."""
        return self.A // 2

    @property
    def offsets_bits(self) -> int:
        return 64 if self.offsets.dtype == np.int64 else 32

    def with_offsets(self, bits: int) -> "Graph":
        dt = np.int64 if bits == 64 else np.int32
        if bits == 32 and self.A >= 2**31:
            raise ValueError("graph too large for int32 offsets")
        return Graph(self.name, self.n, np.ascontiguousarray(self.offsets.astype(dt)),
                     self.cols, self.root, dict(self.meta))


# ---------------------------------------------------------------- primitives

def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded Fisher-Yates permutation; out[i] = new id of vertex i."""
    out = np.empty(n, dtype=np.int32)
    _gen().gg_permutation(n, seed, _ptr(out))
    return out


def uniform(k: int, bound: int, seed: int) -> np.ndarray:
    """k counter-based uniform integers in [0, bound)."""
    out = np.empty(k, dtype=np.int64)
    if k:
        _gen().gg_uniform(k, bound, seed, _ptr(out))
    return out


def from_edges(n: int, u, v, name: str = "edges", root: int = 0,
               offsets_bits: int = 32, meta: dict | None = None) -> Graph:
    """Pack an undirected edge list into the library's CSR contract."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.int32))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    m = int(u.shape[0])
    off = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    A = _gen().gg_build_csr(n, m, _ptr(u), _ptr(v), _ptr(off), _ptr(cols))
    if A < 0:
        raise ValueError("edge endpoint out of range")
    cols = np.ascontiguousarray(cols[:A]).copy()
    if offsets_bits == 32:
        if A >= 2**31:
            raise ValueError("graph too large for int32 offsets")
        off = off.astype(np.int32)
    return Graph(name, n, off, cols, root, meta or {})


# ---------------------------------------------------------------- families

def grid(W: int, H: int, seed: int = 1, permute: bool = True, root: str | int = "corner",
         offsets_bits: int = 32) -> Graph:
    """W x H 4-neighbour grid; vertex (i, j) has id i*W + j before permutation.

    root = "corner" picks the (permuted) id of corner (0, 0); "random" a seeded
    uniform vertex; an int is taken as is (an id after permutation).
    """
    n = W * H
    idx = np.arange(n, dtype=np.int64).reshape(H, W)
    hu = idx[:, :-1].ravel(); hv = idx[:, 1:].ravel()
    vu = idx[:-1, :].ravel(); vv = idx[1:, :].ravel()
    u = np.concatenate([hu, vu]); v = np.concatenate([hv, vv])
    if permute:
        pi = permutation(n, seed).astype(np.int64)
        u = pi[u]; v = pi[v]
    else:
        pi = np.arange(n, dtype=np.int64)
    if root == "corner":
        r = int(pi[0])
    elif root == "random":
        r = int(uniform(1, n, seed + 7777)[0])
    else:
        r = int(root)
    return from_edges(n, u, v, name=f"grid{W}x{H}", root=r, offsets_bits=offsets_bits,
                      meta={"family": "grid", "W": W, "H": H, "seed": seed, "permuted": permute})


def chain_chords(n: int, density: float, seed: int = 1, permute: bool = True,
                 offsets_bits: int = 32) -> Graph:
    """Path 0-1-...-(n-1) plus round(density*n) uniformly random chords.

    Chords that repeat a path edge, another chord or are self-loops are
    dropped by the CSR packing, so the stored chord count can be slightly
    lower. Ids are permuted by seed when `permute` is set.
    """
    k = int(round(density * n))
    pu = np.arange(n - 1, dtype=np.int64); pv = pu + 1
    cu = uniform(k, n, seed * 2 + 1); cv = uniform(k, n, seed * 2 + 2)
    u = np.concatenate([pu, cu]); v = np.concatenate([pv, cv])
    if permute:
        pi = permutation(n, seed).astype(np.int64)
        u = pi[u]; v = pi[v]
        r = int(pi[0])
    else:
        r = 0
    return from_edges(n, u, v, name=f"chain{n}_d{density:g}", root=r, offsets_bits=offsets_bits,
                      meta={"family": "chain", "density": density, "seed": seed})


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 3, connect: bool = True, offsets_bits: int = 64) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale edge draws.

    Symmetrised, self-loops and duplicates removed. With `connect`, every
    component that does not contain vertex 0 gets one edge from its minimum
    vertex id to vertex 0. Root 0, ids not permuted.
    """
    n = 1 << scale
    m = edge_factor * n
    u = np.empty(m, dtype=np.int32); v = np.empty(m, dtype=np.int32)
    _gen().gg_rmat_edges(scale, m, a, b, c, seed, _ptr(u), _ptr(v))
    extra = 0
    if connect:
        eu = np.empty(n, dtype=np.int32); ev = np.empty(n, dtype=np.int32)
        k = _gen().gg_connect_to_zero(n, m, _ptr(u), _ptr(v), _ptr(eu), _ptr(ev))
        extra = int(k)
        u = np.concatenate([u, eu[:k]]); v = np.concatenate([v, ev[:k]])
    return from_edges(n, u, v, name=f"rmat{scale}_ef{edge_factor}", root=0,
                      offsets_bits=offsets_bits,
                      meta={"family": "rmat", "scale": scale, "edge_factor": edge_factor,
                            "seed": seed, "connect_edges": extra})


def random_4regular(n: int, seed: int = 1, offsets_bits: int = 32, max_tries: int = 200) -> Graph:
    """Union of two random Hamiltonian cycles, redrawn until the union is simple."""
    if n < 5:
        raise ValueError("random_4regular needs n >= 5")
    c1 = permutation(n, seed * 1000 + 1).astype(np.int64)
    e1u, e1v = c1, np.roll(c1, -1)
    key1 = np.minimum(e1u, e1v) * n + np.maximum(e1u, e1v)
    key1.sort()
    for t in range(max_tries):
        c2 = permutation(n, seed * 1000 + 2 + t).astype(np.int64)
        e2u, e2v = c2, np.roll(c2, -1)
        key2 = np.minimum(e2u, e2v) * n + np.maximum(e2u, e2v)
        pos = np.searchsorted(key1, key2)
        pos = np.minimum(pos, n - 1)
        if not np.any(key1[pos] == key2):
            u = np.concatenate([e1u, e2u]); v = np.concatenate([e1v, e2v])
            g = from_edges(n, u, v, name=f"reg4_{n}", root=int(uniform(1, n, seed)[0]),
                           offsets_bits=offsets_bits, meta={"family": "reg4", "seed": seed})
            assert g.A == 4 * n
            return g
    raise RuntimeError("could not draw a simple 4-regular graph")


def erdos_renyi(n: int, m: int, seed: int = 1, offsets_bits: int = 32) -> Graph:
    """m uniform random edge draws on n vertices (possibly disconnected)."""
    u = uniform(m, n, seed * 2 + 11); v = uniform(m, n, seed * 2 + 12)
    return from_edges(n, u, v, name=f"er{n}_{m}", root=int(uniform(1, n, seed + 5)[0]) if n else 0,
                      offsets_bits=offsets_bits, meta={"family": "er", "seed": seed})


# ---------------------------------------------------------------- named workloads

def workload_grid256(seed: int = 1) -> Graph:
    """256x256 grid, ids permuted by seed, root = permuted id of corner (0,0)."""
    return grid(256, 256, seed=seed, permute=True, root="corner")


def workload_grid4096(seed: int = 2) -> Graph:
    """4096x4096 grid (16,777,216 vertices, 33,546,240 edges), permuted ids,
    seeded random root."""
    return grid(4096, 4096, seed=seed, permute=True, root="random")


def workload_rmat24(seed: int = 3) -> Graph:
    """R-MAT scale 24, edge factor 16, (0.57, 0.19, 0.19, 0.05), connected to 0,
    int64 offsets, root 0."""
    return rmat(24, 16, 0.57, 0.19, 0.19, seed=seed, connect=True, offsets_bits=64)


# ---------------------------------------------------------------- batches

@dataclass
class Batch:
    """Disjoint graphs packed for rst_build_batch.

    offsets: the graphs' LOCAL offset arrays concatenated (graph g's n_g + 1
    entries start at vtx_off[g] + g); cols: the graphs' LOCAL column arrays
    concatenated; vtx_off / arc_off: int64 prefix sums of vertex and arc
    counts (length G+1); roots: local root of each graph.
    """

    graphs: list
    offsets: np.ndarray
    cols: np.ndarray
    vtx_off: np.ndarray
    arc_off: np.ndarray
    roots: np.ndarray

    @property
    def G(self) -> int:
        return len(self.graphs)

    @property
    def N(self) -> int:
        return int(self.vtx_off[-1])

    @property
    def A(self) -> int:
        return int(self.arc_off[-1])

    @property
    def m(self) -> int:
        return self.A // 2

    @property
    def offsets_bits(self) -> int:
        return 64 if self.offsets.dtype == np.int64 else 32

    def graph_offsets(self, g: int) -> np.ndarray:
        v0 = int(self.vtx_off[g]) + g
        return self.offsets[v0:v0 + self.graphs[g].n + 1]

    def graph_cols(self, g: int) -> np.ndarray:
        return self.cols[int(self.arc_off[g]):int(self.arc_off[g + 1])]


def pack_batch(graphs, offsets_bits: int = 32) -> Batch:
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    arc_off = np.zeros(G + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        vtx_off[i + 1] = vtx_off[i] + g.n
        arc_off[i + 1] = arc_off[i] + g.A
    N, A = int(vtx_off[-1]), int(arc_off[-1])
    dt = np.int64 if offsets_bits == 64 else np.int32
    offsets = np.empty(N + G, dtype=dt)
    cols = np.empty(A, dtype=np.int32)
    for i, g in enumerate(graphs):
        v0, a0 = int(vtx_off[i]) + i, int(arc_off[i])
        offsets[v0:v0 + g.n + 1] = g.offsets.astype(dt)
        cols[a0:a0 + g.A] = g.cols
    roots = np.array([g.root for g in graphs], dtype=np.int32)
    return Batch(list(graphs), offsets, cols, vtx_off, arc_off, roots)


def batch_graph_family(i: int, seed: int, n: int) -> Graph:
    """One member of a mixed batch: grid / chain+chords / R-MAT by i mod 3.

    Sizes and shape knobs are drawn from a counter-based stream of (seed, i).
    """
    r = uniform(4, 1 << 30, seed * 1_000_003 + i)
    fam = i % 3
    gseed = int(seed * 100_003 + i)
    if fam == 0:
        # aspect ratio log-uniform in [1, 1024]
        aspect = math.exp(r[0] / (1 << 30) * math.log(1024.0))
        H = max(1, int(round(math.sqrt(n / aspect))))
        W = max(1, n // H)
        g = grid(W, H, seed=gseed, permute=True, root="random")
    elif fam == 1:
        d = math.exp(math.log(1e-5) + r[1] / (1 << 30) * (math.log(1e-2) - math.log(1e-5)))
        g = chain_chords(n, d, seed=gseed)
        g.root = int(uniform(1, n, gseed + 3)[0])
    else:
        scale = max(10, min(18, int(round(math.log2(n)))))
        g = rmat(scale, 16, seed=gseed, connect=True, offsets_bits=32)
    return g


def batch_sizes(G: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """G vertex counts log-uniform in [lo, hi]."""
    r = uniform(G, 1 << 30, seed * 7 + 1).astype(np.float64) / (1 << 30)
    return np.exp(np.log(lo) + r * (np.log(hi) - np.log(lo))).astype(np.int64)


def workload_batch(G: int = 4096, lo: int = 1024, hi: int = 4096, seed: int = 4) -> Batch:
    """Mixed batch: G graphs, vertex counts log-uniform in [lo, hi], families in
    turn grid (aspect 1-1024) / chain with chords (density 1e-5..1e-2) / R-MAT
    (scale ~log2 n, connected), one seeded root per graph."""
    sizes = batch_sizes(G, lo, hi, seed)
    return pack_batch([batch_graph_family(i, seed, int(n)) for i, n in enumerate(sizes)])
