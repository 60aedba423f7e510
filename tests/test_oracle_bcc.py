"""Pins of the biconnected-components oracle (Hopcroft-Tarjan depth-first
search), from definitions it does not use:

* brute force on tiny multigraphs: an edge set is a simple cycle iff it is
  connected and every vertex it touches has degree two in it; two edges share
  a block iff a chain of simple cycles links them; an edge on no cycle is a
  block by itself; v is a cut vertex iff its neighbours fall into two or more
  components of G - v;
* closed forms (cycle, path, star, bowtie, grid, complete graph, two cycles
  joined by a bridge);
* networkx's biconnected components and articulation points, where installed.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

NONE = 0xFFFFFFFF


def _csr_from_multiedges(n, edges):
    """CSR with sorted rows; every undirected edge (u, v) gives arcs u->v and
    v->u (a self-loop gives the single arc u->u twice, as in a symmetric CSR)."""
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        rows[v].append(u)
    off = np.zeros(n + 1, dtype=np.int64)
    for i in range(n):
        rows[i].sort()
        off[i + 1] = off[i] + len(rows[i])
    col = np.array([w for r in rows for w in r], dtype=np.int32)
    return off, col


def _brute_force(n, edges, off, col):
    m = len(edges)
    parent = list(range(m))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    real = [i for i, (u, v) in enumerate(edges) if u != v]
    for k in range(2, len(real) + 1):
        for sub in itertools.combinations(real, k):
            deg = {}
            for i in sub:
                u, v = edges[i]
                deg[u] = deg.get(u, 0) + 1
                deg[v] = deg.get(v, 0) + 1
            if any(d != 2 for d in deg.values()):
                continue
            # connected?
            verts = list(deg)
            seen = {verts[0]}
            stack = [verts[0]]
            while stack:
                x = stack.pop()
                for i in sub:
                    u, v = edges[i]
                    for a, b in ((u, v), (v, u)):
                        if a == x and b not in seen:
                            seen.add(b)
                            stack.append(b)
            if len(seen) != len(verts):
                continue
            for i in sub[1:]:
                ra, rb = find(sub[0]), find(i)
                if ra != rb:
                    parent[rb] = ra
    # block label: smallest CSR position among the block's arcs
    def positions(u, v):
        return [a for a in range(off[u], off[u + 1]) if col[a] == v]

    blocks = {}
    for i in real:
        u, v = edges[i]
        blocks.setdefault(find(i), set()).update(positions(u, v) + positions(v, u))
    lab_of_block = {b: min(p) for b, p in blocks.items()}
    label = np.full(len(col), NONE, dtype=np.uint64)
    for i in real:
        u, v = edges[i]
        for a in positions(u, v) + positions(v, u):
            label[a] = lab_of_block[find(i)]
    # cut vertices by deletion
    cut = np.zeros(n, dtype=np.uint8)
    for x in range(n):
        nb = sorted({w for w in col[off[x]:off[x + 1]] if w != x})
        if len(nb) < 2:
            continue
        comp = {}
        for s in nb:
            if s in comp:
                continue
            comp[s] = s
            stack = [s]
            while stack:
                y = stack.pop()
                for w in col[off[y]:off[y + 1]]:
                    w = int(w)
                    if w != x and w not in comp:
                        comp[w] = s
                        stack.append(w)
        if len({comp[s] for s in nb}) > 1:
            cut[x] = 1
    return label.astype(np.uint32), cut, len(blocks)


@pytest.mark.parametrize("seed", range(40))
def test_bcc_brute_force_tiny_multigraphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(0, 11))
    edges = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
    if seed % 3 == 0:  # mostly simple graphs, some multigraphs with loops
        edges = [(u, v) for u, v in {(min(a, b), max(a, b)) for a, b in edges} if u != v]
    off, col = _csr_from_multiedges(n, edges)
    lab, cut, nb = oracle.bcc(n, off, col)
    blab, bcut, bnb = _brute_force(n, edges, off, col)
    assert np.array_equal(lab, blab), (edges, lab, blab)
    assert np.array_equal(cut, bcut), (edges, cut, bcut)
    assert nb == bnb


def _simple(n, pairs):
    return _csr_from_multiedges(n, pairs)


def test_bcc_closed_forms():
    # cycle C_6: one block, no cut vertex
    off, col = _simple(6, [(i, (i + 1) % 6) for i in range(6)])
    lab, cut, nb = oracle.bcc(6, off, col)
    assert nb == 1 and set(lab.tolist()) == {0} and cut.sum() == 0
    # path P_5: four bridges, internal vertices cut
    off, col = _simple(5, [(i, i + 1) for i in range(4)])
    lab, cut, nb = oracle.bcc(5, off, col)
    assert nb == 4 and cut.tolist() == [0, 1, 1, 1, 0]
    # star K_{1,4}: four blocks, the centre is the only cut vertex
    off, col = _simple(5, [(0, k) for k in range(1, 5)])
    lab, cut, nb = oracle.bcc(5, off, col)
    assert nb == 4 and cut.tolist() == [1, 0, 0, 0, 0]
    # K_4: one block
    off, col = _simple(4, [(a, b) for a in range(4) for b in range(a + 1, 4)])
    lab, cut, nb = oracle.bcc(4, off, col)
    assert nb == 1 and cut.sum() == 0
    # two triangles joined by the bridge 2-3: three blocks, cut vertices 2 and 3
    off, col = _simple(6, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 5), (3, 5)])
    lab, cut, nb = oracle.bcc(6, off, col)
    assert nb == 3 and cut.tolist() == [0, 0, 1, 1, 0, 0]
    # a doubled edge is a 2-cycle: one block
    off, col = _csr_from_multiedges(2, [(0, 1), (0, 1)])
    lab, cut, nb = oracle.bcc(2, off, col)
    assert nb == 1 and lab.tolist() == [0, 0, 0, 0]


@pytest.mark.parametrize("W,H", [(2, 2), (5, 3), (7, 7)])
def test_bcc_grid_is_one_block(W, H):
    g = graphs.grid(W, H, seed=3, permute=True)
    lab, cut, nb = oracle.bcc(g.n, g.offsets, g.cols)
    assert nb == 1 and cut.sum() == 0 and set(lab.tolist()) == {0}


@pytest.mark.parametrize("seed", range(6))
def test_bcc_matches_networkx(seed):
    nx = pytest.importorskip("networkx")
    g = (graphs.erdos_renyi(300, 330, seed=seed) if seed % 2 == 0
         else graphs.chain_chords(400, 0.01, seed=seed))
    lab, cut, nb = oracle.bcc(g.n, g.offsets, g.cols)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, g.cols) if a < b)
    comps = list(nx.biconnected_component_edges(G))
    assert nb == len(comps)
    pos = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(src, g.cols))}
    for comp in comps:
        arcs = [pos[(a, b)] for a, b in comp] + [pos[(b, a)] for a, b in comp]
        assert len({int(lab[a]) for a in arcs}) == 1
        assert int(lab[arcs[0]]) == min(arcs)
    art = set(nx.articulation_points(G))
    assert set(np.nonzero(cut)[0].tolist()) == art
