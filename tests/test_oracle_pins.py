"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: hand-derived
fixtures (tests/golden), closed forms, brute-force enumeration on tiny
graphs, Kirchhoff's matrix-tree theorem, an independent library routine
(scipy's connected components), an independent rotation-rule DFS, and
invariants of Euler tours.  A plausible slip in the oracle (a swapped parent
rule, a dropped wrap-around, an off-by-one in the cycle break, a wrong key
order) fails at least one of them.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_2603_11645_gb300 import graphs

pytestmark = pytest.mark.filterwarnings("ignore")


def G(n, edges, root=0):
    u = [a for a, b in edges]
    v = [b for a, b in edges]
    return graphs.from_edges(n, u, v, root=root)


def sorted_arcs_with_rank(n, tu, tv, root):
    s, d, r, p = oracle.euler_tour(n, tu, tv, root)
    return [(int(a), int(b), int(c)) for a, b, c in zip(s, d, r)], p


# ------------------------------------------------------------------ golden fixtures

@pytest.mark.parametrize("name,n,edges,root", [
    ("path5_root0.txt", 5, [(0, 1), (1, 2), (2, 3), (3, 4)], 0),
    ("star6_root3.txt", 6, [(0, j) for j in range(1, 6)], 3),
    ("star6_root0.txt", 6, [(0, j) for j in range(1, 6)], 0),
])
def test_euler_golden(name, n, edges, root):
    gold = load_golden(name)
    tu = [a for a, b in edges]
    tv = [b for a, b in edges]
    arcs, parent = sorted_arcs_with_rank(n, tu, tv, root)
    assert arcs == [tuple(x) for x in gold["arcs"]]
    assert parent.tolist() == gold["parent"][0]
    assert oracle.root_forest(n, tu, tv, root).tolist() == gold["parent"][0]


def test_grid_comb_golden():
    gold = load_golden("grid4x3_comb.txt")
    g = graphs.grid(4, 3, permute=False, root=0)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert [[int(a), int(b)] for a, b in zip(tu, tv)] == gold["tree"]
    assert oracle.rst(g.n, g.offsets, g.cols, 0).tolist() == gold["parent"][0]
    lev, par = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert lev.tolist() == gold["level"][0]


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [2, 3, 7, 64, 1000])
def test_path_closed_form(n):
    edges = [(i, i + 1) for i in range(n - 1)]
    g = G(n, edges)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    assert len(tu) == n - 1 and (lab == 0).all()
    arcs, parent = sorted_arcs_with_rank(n, tu, tv, 0)
    assert parent.tolist() == [0] + list(range(n - 1))
    for s, d, r in arcs:
        if d == s + 1:
            assert r == s
        else:
            assert r == 2 * (n - 1) - 1 - d


@pytest.mark.parametrize("k", [1, 2, 5, 40])
def test_star_closed_form(k):
    n = k + 1
    tu, tv = [0] * k, list(range(1, n))
    arcs, parent = sorted_arcs_with_rank(n, tu, tv, 0)
    for s, d, r in arcs:
        if s == 0:
            assert r == 2 * (d - 1)
        else:
            assert r == 2 * s - 1
    # rooted at each leaf: the tour starts with (l,0), then wraps through the centre
    for leaf in range(1, n):
        arcs, parent = sorted_arcs_with_rank(n, tu, tv, leaf)
        order = [None] * (2 * k)
        for s, d, r in arcs:
            order[r] = (s, d)
        expect = [(leaf, 0)]
        for j in list(range(leaf + 1, n)) + list(range(1, leaf)):
            expect += [(0, j), (j, 0)]
        expect.append((0, leaf))
        assert order == expect
        assert parent[0] == leaf and parent[leaf] == leaf


@pytest.mark.parametrize("W,H", [(4, 3), (1, 9), (9, 1), (17, 5)])
def test_grid_comb_and_manhattan(W, H):
    g = graphs.grid(W, H, permute=False, root=0)
    par = oracle.rst(g.n, g.offsets, g.cols, 0)
    lev, bpar = oracle.bfs(g.n, g.offsets, g.cols, 0)
    for i in range(H):
        for j in range(W):
            v = i * W + j
            assert lev[v] == i + j
            if v == 0:
                assert par[v] == 0
            elif i == 0:
                assert par[v] == v - 1 and bpar[v] == v - 1
            else:
                assert par[v] == v - W and bpar[v] == v - W


# ------------------------------------------------------------------ brute force

def _brute_msf(n, edges):
    keys = sorted({(min(a, b), max(a, b)) for a, b in edges if a != b})
    # number of components by union-find
    p = list(range(n))

    def f(x):
        while p[x] != x:
            x = p[x]
        return x
    for a, b in keys:
        ra, rb = f(a), f(b)
        if ra != rb:
            p[ra] = rb
    c = len({f(x) for x in range(n)})
    best, best_w = None, None
    rank_of = {e: i for i, e in enumerate(keys)}
    for sub in itertools.combinations(keys, n - c):
        q = list(range(n))

        def g_(x):
            while q[x] != x:
                x = q[x]
            return x
        ok = True
        for a, b in sub:
            ra, rb = g_(a), g_(b)
            if ra == rb:
                ok = False
                break
            q[ra] = rb
        if not ok:
            continue
        w = sum(2 ** rank_of[e] for e in sub)  # lexicographic minimum over sorted keys
        if best_w is None or w < best_w:
            best, best_w = sorted(sub), w
    return best


@pytest.mark.parametrize("seed", range(40))
def test_kruskal_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    m = int(rng.integers(0, min(13, n * (n - 1) // 2) + 1))
    edges = [tuple(int(x) for x in rng.integers(0, n, 2)) for _ in range(m)]
    g = G(n, edges)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    want = _brute_msf(n, edges)
    assert sorted(zip(tu.tolist(), tv.tolist())) == want
    # unique MSF under distinct weights: every other spanning forest weighs more
    assert len(tu) == len(want)


def _floyd(n, edges):
    INF = 10 ** 9
    D = [[0 if i == j else INF for j in range(n)] for i in range(n)]
    for a, b in edges:
        if a != b:
            D[a][b] = D[b][a] = 1
    for k in range(n):
        for i in range(n):
            for j in range(n):
                if D[i][k] + D[k][j] < D[i][j]:
                    D[i][j] = D[i][k] + D[k][j]
    return D


@pytest.mark.parametrize("seed", range(30))
def test_bfs_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 14))
    edges = [tuple(int(x) for x in rng.integers(0, n, 2)) for _ in range(m)]
    root = int(rng.integers(0, n))
    g = G(n, edges, root)
    lev, par = oracle.bfs(n, g.offsets, g.cols, root)
    D = _floyd(n, edges)
    INF = 10 ** 9
    # sources: root, then the minimum id of every other component
    src = [None] * n
    for v in range(n):
        if D[root][v] < INF:
            src[v] = root
    for v in range(n):
        if src[v] is None:
            for w in range(n):
                if D[v][w] < INF and src[w] is None:
                    src[w] = v
    nbr = {v: set() for v in range(n)}
    for a, b in edges:
        if a != b:
            nbr[a].add(b)
            nbr[b].add(a)
    for v in range(n):
        assert lev[v] == D[src[v]][v]
        if v == src[v]:
            assert par[v] == v
        else:
            cands = [u for u in nbr[v] if D[src[v]][u] == D[src[v]][v] - 1]
            assert par[v] == min(cands)


# ------------------------------------------------------------------ Kirchhoff

def _det(M):
    M = [[Fraction(x) for x in row] for row in M]
    n = len(M)
    det = Fraction(1)
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] != 0), None)
        if piv is None:
            return 0
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det *= M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            for k in range(c, n):
                M[r][k] -= f * M[c][k]
    return int(det)


@pytest.mark.parametrize("n,edges", [
    (4, [(0, 1), (1, 2), (2, 3), (3, 0)]),
    (5, [(a, b) for a in range(5) for b in range(a + 1, 5)]),
    (6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (1, 4)]),
    (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
])
def test_verifier_counts_spanning_trees(n, edges):
    g = G(n, edges)
    L = [[0] * n for _ in range(n)]
    for a, b in {(min(a, b), max(a, b)) for a, b in edges}:
        L[a][a] += 1
        L[b][b] += 1
        L[a][b] -= 1
        L[b][a] -= 1
    trees = _det([row[1:] for row in L[1:]])
    for root in (0, n - 1):
        accepted = 0
        for P in itertools.product(range(n), repeat=n):
            if oracle.verify(n, g.offsets, g.cols, root, np.array(P, np.int32)) == oracle.VALID:
                accepted += 1
        assert accepted == trees


# ------------------------------------------------------------------ verifier mutations

def _families():
    yield graphs.grid(9, 7, seed=3)
    yield graphs.chain_chords(300, 0.05, seed=4)
    yield graphs.erdos_renyi(200, 150, seed=5)          # disconnected
    yield graphs.rmat(8, 4, seed=6, connect=False, offsets_bits=32)
    yield graphs.random_4regular(100, seed=7)


@pytest.mark.parametrize("gi", range(5))
def test_verifier_mutations(gi):
    g = list(_families())[gi]
    n = g.n
    par = oracle.rst(n, g.offsets, g.cols, g.root)
    assert oracle.verify(n, g.offsets, g.cols, g.root, par) == oracle.VALID
    rng = np.random.default_rng(gi)
    nonroot = [v for v in range(n) if par[v] != v]
    v = int(rng.choice(nonroot))
    # 1: root not self
    p = par.copy(); p[g.root] = par[v] if par[v] != g.root else v
    if p[g.root] != g.root:
        assert oracle.verify(n, g.offsets, g.cols, g.root, p) == oracle.BAD_ROOT
    # 2: parent out of range
    p = par.copy(); p[v] = n
    assert oracle.verify(n, g.offsets, g.cols, g.root, p) == oracle.PARENT_RANGE
    # 3: non-edge parent
    row = set(g.cols[g.offsets[v]:g.offsets[v + 1]].tolist())
    w = next(x for x in range(n) if x != v and x not in row)
    p = par.copy(); p[v] = w
    assert oracle.verify(n, g.offsets, g.cols, g.root, p) == oracle.NON_EDGE
    # 4: a 2-cycle through a tree edge
    u = int(par[v])
    p = par.copy(); p[u] = v
    if u != g.root:
        assert oracle.verify(n, g.offsets, g.cols, g.root, p) == oracle.CYCLE
    # 5: cut a subtree loose
    p = par.copy(); p[v] = v
    assert oracle.verify(n, g.offsets, g.cols, g.root, p) == oracle.NOT_SPANNING


def test_verifier_component_root_rule():
    g = graphs.erdos_renyi(60, 40, seed=9)
    lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    par = oracle.root_forest(g.n, tu, tv, g.root)
    comps = {}
    for v in range(g.n):
        comps.setdefault(int(lab[v]), []).append(v)
    big = next(c for c, vs in comps.items() if len(vs) >= 2 and c != lab[g.root])
    other = max(comps[big])
    # reroot that component at a vertex that is not its minimum
    sub_u = [a for a, b in zip(tu, tv) if lab[a] == big]
    sub_v = [b for a, b in zip(tu, tv) if lab[a] == big]
    pr = oracle.root_forest(g.n, sub_u, sub_v, other)
    p = par.copy()
    for x in comps[big]:
        p[x] = pr[x]
    assert oracle.verify(g.n, g.offsets, g.cols, g.root, p, strict_roots=False) == oracle.VALID
    assert oracle.verify(g.n, g.offsets, g.cols, g.root, p) == oracle.COMPONENT_ROOT


# ------------------------------------------------------------------ independent algorithms

def test_labels_match_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for g in _families():
        lab, tu, tv = oracle.cc_kruskal(g.n, g.offsets, g.cols)
        mat = sp.csr_matrix((np.ones(g.A), g.cols, g.offsets.astype(np.int64)), shape=(g.n, g.n))
        c, sl = csgraph.connected_components(mat, directed=False)
        assert len(tu) == g.n - c
        mins = {}
        for v in range(g.n):
            mins.setdefault(sl[v], v)
        assert all(lab[v] == mins[sl[v]] for v in range(g.n))


def _rotation_dfs(n, tu, tv, r):
    adj = {v: [] for v in range(n)}
    for a, b in zip(tu, tv):
        adj[int(a)].append(int(b))
        adj[int(b)].append(int(a))
    for v in adj:
        adj[v].sort()
    tour = []
    import sys
    sys.setrecursionlimit(10000)

    def visit(v, p):
        nb = adj[v]
        if p is None:
            order = nb
        else:
            k = nb.index(p)
            order = nb[k + 1:] + nb[:k]
        for c in order:
            tour.append((v, c))
            visit(c, v)
            tour.append((c, v))
    visit(r, None)
    return tour


@pytest.mark.parametrize("seed", range(12))
def test_euler_equals_rotation_dfs(seed):
    """The succ equation walks the same tour as a DFS that, entering v from p,
    continues with the neighbours after p in v's sorted order, cyclically."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 120))
    # random tree: attach each vertex to an earlier one, then relabel
    pi = rng.permutation(n)
    tu = [int(pi[i]) for i in range(1, n)]
    tv = [int(pi[int(rng.integers(0, i))]) for i in range(1, n)]
    root = int(rng.integers(0, n))
    arcs, parent = sorted_arcs_with_rank(n, tu, tv, root)
    order = [None] * (2 * (n - 1))
    for s, d, r in arcs:
        order[r] = (s, d)
    assert order == _rotation_dfs(n, tu, tv, root)


@pytest.mark.parametrize("gi", range(5))
def test_euler_invariants(gi):
    g = list(_families())[gi]
    n = g.n
    lab, tu, tv = oracle.cc_kruskal(n, g.offsets, g.cols)
    s, d, r, par = oracle.euler_tour(n, tu, tv, g.root)
    assert np.array_equal(par, oracle.root_forest(n, tu, tv, g.root))
    # sorted order
    key = s.astype(np.int64) * n + d
    assert np.all(np.diff(key) > 0)
    # per tree: ranks are a permutation of 0..2(size-1)-1
    size = np.bincount(lab, minlength=n)
    by_tree = {}
    for a, rk in zip(s, r):
        by_tree.setdefault(int(lab[a]), []).append(int(rk))
    for t, rks in by_tree.items():
        assert sorted(rks) == list(range(2 * (size[t] - 1)))
    # down arc before up arc; subtree size from ranks
    pos = {(int(a), int(b)): int(k) for a, b, k in zip(s, d, r)}
    sub = np.ones(n, np.int64)
    order = np.argsort(-oracle.bfs(n, g.offsets, g.cols, g.root)[0])  # not needed for sizes
    del order
    # subtree sizes by repeated accumulation from leaves
    children = {v: [] for v in range(n)}
    for v in range(n):
        if par[v] != v:
            children[int(par[v])].append(v)
    import sys
    sys.setrecursionlimit(100000)

    def size_of(v):
        tot, stack, seen = 0, [v], []
        while stack:
            x = stack.pop()
            tot += 1
            stack.extend(children[x])
        return tot
    for v in range(n):
        if par[v] != v:
            down, up = pos[(int(par[v]), v)], pos[(v, int(par[v]))]
            assert down < up
            assert (up - down + 1) // 2 == size_of(v)
    del sub


# ------------------------------------------------------------------ PR-RST

def test_prrst_golden():
    gold = load_golden("prrst_path4_root3.txt")
    g = G(4, [(0, 2), (1, 2), (1, 3)], root=3)
    par, rounds = oracle.prrst(4, g.offsets, g.cols, 3)
    assert par.tolist() == gold["parent"][0]
    assert rounds == gold["rounds"][0][0]


@pytest.mark.parametrize("gi", range(5))
def test_prrst_is_a_valid_rst(gi):
    """PR-RST fixes no unique tree; its output must pass the exact verifier
    (root rule for other components included) and the round count must stay
    logarithmic."""
    g = list(_families())[gi]
    par, rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    assert oracle.verify(g.n, g.offsets, g.cols, g.root, par) == oracle.VALID
    assert rounds <= 4 * int(np.ceil(np.log2(g.n + 1))) + 2


def test_prrst_path_and_star():
    n = 9
    g = G(n, [(i, i + 1) for i in range(n - 1)], root=4)
    par, _ = oracle.prrst(n, g.offsets, g.cols, 4)
    assert par.tolist() == [1, 2, 3, 4, 4, 4, 5, 6, 7]
    g = G(n, [(0, j) for j in range(1, n)], root=5)
    par, _ = oracle.prrst(n, g.offsets, g.cols, 5)
    assert par.tolist() == [5] + [0] * 4 + [5] + [0] * 3


def _prrst_pin_graphs():
    yield from _families()
    yield graphs.grid(30, 20, seed=8)
    yield graphs.erdos_renyi(500, 1500, seed=9)
    yield graphs.rmat(9, 8, seed=10, connect=True, offsets_bits=32)


def _tree_edge_set(par):
    return {(min(v, int(p)), max(v, int(p))) for v, p in enumerate(par) if p != v}


@pytest.mark.parametrize("gi", range(8))
def test_prrst_keeps_the_first_two_rounds_grafts(gi):
    """Grafting only adds edges and path reversal only turns them around, so
    the final tree contains every edge the first two rounds graft, and those
    follow from the round rules alone (Section III-C, reading R9).
    Round 0 (minimum rule) on singletons: every vertex with a smaller
    neighbour grafts onto its smallest neighbour.  The trees after it are the
    components of those edges, each rooted at its smallest vertex (the grafts
    follow decreasing ids).  Round 1 (maximum rule): each such tree grafts along
    its smallest arc (u, v) (u in the tree) into a tree with a larger root.
    A swapped rule, a reversed key order or a graft that loses an edge fails
    here; the components come from scipy, not from the oracle's pointers."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    g = list(_prrst_pin_graphs())[gi]
    n = g.n
    par, rounds = oracle.prrst(n, g.offsets, g.cols, g.root)
    tree = _tree_edge_set(par)
    off = g.offsets.astype(np.int64)
    src = np.repeat(np.arange(n), np.diff(off))
    dst = g.cols.astype(np.int64)
    # round 0
    smaller = dst < src
    minnbr = np.full(n, -1)
    for u, v in zip(src[smaller], dst[smaller]):
        if minnbr[u] < 0 or v < minnbr[u]:
            minnbr[u] = v
    r0 = [(int(min(v, m)), int(max(v, m))) for v, m in enumerate(minnbr) if m >= 0]
    assert set(r0) <= tree
    # trees after round 0 and their roots (smallest vertex)
    has = minnbr >= 0
    a = coo_matrix((np.ones(has.sum()), (np.arange(n)[has], minnbr[has])), shape=(n, n))
    _, comp = connected_components(a, directed=False)
    root_of_comp = np.full(comp.max() + 1, n)
    np.minimum.at(root_of_comp, comp, np.arange(n))
    rt = root_of_comp[comp]
    # round 1: smallest (u, v) with u in the tree and a larger root across the arc
    elig = rt[dst] > rt[src]
    best = {}
    for u, v in zip(src[elig], dst[elig]):
        c = comp[u]
        if c not in best or (u, v) < best[c]:
            best[c] = (int(u), int(v))
    r1 = {(min(u, v), max(u, v)) for u, v in best.values()}
    assert r1 <= tree
    assert len(tree) >= len(set(r0) | r1)


def _prrst_by_components(n, offsets, cols, init=None):
    """PR-RST's tree edges and round count, derived from the round rules at
    the level of whole trees (no parent pointers, no path reversal): in round
    t every tree with an arc into a tree of smaller (t even) or larger (t odd)
    root grafts along its smallest such arc (u, v), u in the tree; a graft
    re-roots the tree at u, so the merged tree keeps the root of the tree at
    the end of the graft chain.  Stops after the first round without a graft."""
    off = np.asarray(offsets, dtype=np.int64)
    src = np.repeat(np.arange(n), np.diff(off))
    dst = np.asarray(cols, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    edges = set()
    root = np.arange(n)
    if init is not None:
        init = np.asarray(init, dtype=np.int64)
        for v in range(n):
            x = v
            while init[x] != x:
                x = init[x]
            root[v] = x
            if init[v] != v:
                edges.add((min(v, int(init[v])), max(v, int(init[v]))))
    t = 0
    while True:
        rs, rd = root[src], root[dst]
        elig = (rd < rs) if t % 2 == 0 else (rd > rs)
        best = {}
        for u, v in zip(src[elig], dst[elig]):
            r = int(root[u])
            if r not in best or (int(u), int(v)) < best[r]:
                best[r] = (int(u), int(v))
        if not best:
            return edges, t + 1
        nxt = {}
        for r, (u, v) in best.items():
            edges.add((min(u, v), max(u, v)))
            nxt[r] = int(root[v])
        sink = {}
        for r in set(root.tolist()):
            x = r
            while x in nxt:
                x = nxt[x]
            sink[r] = x
        root = np.array([sink[int(r)] for r in root])
        t += 1


@pytest.mark.parametrize("gi", range(8))
def test_prrst_edge_set_equals_the_tree_level_derivation(gi):
    """The oracle's PR-RST (pointer-level rounds with path reversal) against
    the same rules applied to whole trees: identical tree edges and round
    count, and the final tree rooted at the requested root (other components
    at their smallest vertex)."""
    g = list(_prrst_pin_graphs())[gi]
    par, rounds = oracle.prrst(g.n, g.offsets, g.cols, g.root)
    edges, want_rounds = _prrst_by_components(g.n, g.offsets, g.cols)
    assert _tree_edge_set(par) == edges
    assert rounds == want_rounds
    lab, _, _ = oracle.cc_kruskal(g.n, g.offsets, g.cols)
    for v in range(g.n):
        is_root = par[v] == v
        want_root = v == g.root or (lab[v] == v and lab[g.root] != v)
        assert is_root == want_root, v


@pytest.mark.parametrize("seed", range(6))
def test_prrst_from_a_forest_equals_the_tree_level_derivation(seed):
    """Edge insertions (rounds started from a rooted forest) against the
    same tree-level derivation started from the forest's trees."""
    rng = np.random.default_rng(40 + seed)
    g = graphs.grid(12, 9, seed=seed + 1)
    n = g.n
    par0 = oracle.rst(n, g.offsets, g.cols, g.root)
    # drop a random third of the tree edges: the rest is the starting forest
    init = par0.copy()
    for v in np.nonzero(rng.random(n) < 0.33)[0]:
        init[v] = v
    # every chain must still end at a root: re-root each piece at its top
    par, rounds = oracle.prrst(n, g.offsets, g.cols, g.root, init=init)
    edges, want_rounds = _prrst_by_components(n, g.offsets, g.cols, init=init)
    assert _tree_edge_set(par) == edges
    assert rounds == want_rounds


# ------------------------------------------------------------------ tree depth

@pytest.mark.parametrize("n,r", [(1, 0), (10, 0), (10, 4), (10, 9)])
def test_tree_depths_path_closed_form(n, r):
    # path 0-1-...-(n-1) rooted at r: depth(i) = |i - r|
    parent = [i + 1 if i < r else (i - 1 if i > r else i) for i in range(n)]
    assert np.array_equal(oracle.tree_depths(n, parent), np.abs(np.arange(n) - r))


def test_tree_depths_star_and_forest():
    # star with centre 0 rooted at leaf 3: the leaf 0, the centre 1, the rest 2
    parent = [3, 0, 0, 3, 0, 0]
    assert list(oracle.tree_depths(6, parent)) == [1, 2, 2, 0, 2, 2]
    # two trees and a singleton
    assert list(oracle.tree_depths(6, [0, 0, 1, 3, 3, 5])) == [0, 1, 2, 0, 1, 0]


@pytest.mark.parametrize("W,H", [(5, 4), (7, 1), (1, 6)])
def test_tree_depths_of_the_grid_comb(W, H):
    # identity-labelled grid rooted at 0: the Kruskal tree is the comb (row 0
    # plus every vertical edge), so vertex (i, j) sits at depth i + j
    g = graphs.grid(W, H, permute=False, root=0)
    par = oracle.rst(g.n, g.offsets, g.cols, 0)
    want = np.array([i + j for i in range(H) for j in range(W)])
    assert np.array_equal(oracle.tree_depths(g.n, par), want)


@pytest.mark.parametrize("seed", range(4))
def test_bfs_tree_depth_is_the_bfs_level(seed):
    # every BFS parent sits one level up, so depth in the BFS tree = level
    g = graphs.erdos_renyi(400, 700, seed=seed)
    lev, par = oracle.bfs(g.n, g.offsets, g.cols, g.root)
    d = oracle.tree_depths(g.n, par)
    reached = lev >= 0
    assert np.array_equal(d[reached], lev[reached])


def test_tree_depths_rejects_cycles_and_range():
    with pytest.raises(ValueError):
        oracle.tree_depths(3, [1, 2, 0])
    with pytest.raises(ValueError):
        oracle.tree_depths(4, [0, 2, 3, 1])  # 1 -> 2 -> 3 -> 1
    with pytest.raises(ValueError):
        oracle.tree_depths(3, [0, 5, 0])
