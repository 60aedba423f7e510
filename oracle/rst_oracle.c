/*
 * CPU oracle for rooted spanning trees (RST).  TEST INFRASTRUCTURE ONLY.
 *
 * Plain, sequential, single-threaded C written from the paper "Beyond BFS: A
 * Comparative Study of Rooted Spanning Tree Algorithms on GPUs"
 * (arXiv 2603.11645).  It shares no code, header, table or helper with the
 * CUDA library; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.
 *
 * Output contract (Section I): the RST is a parent array P with P[r] = r and
 * exactly one parent for every other vertex.  For a disconnected input every
 * component that does not contain r is rooted at its minimum vertex id (the
 * forest generalisation of Section III-D).
 *
 * Functions
 *   or_cc_kruskal   connected components + spanning forest (Section III-B):
 *                   Kruskal over edge keys (min(u,v), max(u,v)) ascending.
 *                   This is the unique minimum spanning forest under those
 *                   distinct keys, which a min-key hooking rule must reproduce.
 *   or_root_forest  parent array of a forest for the given root (plain
 *                   depth-first search; independent of the Euler tour).
 *   or_euler_tour   the Euler-tour rooting of Section III-D executed
 *                   sequentially: lexicographic arc sort, first/last/next,
 *                   the succ equation, cycle breaking at rev(last[r]), a
 *                   sequential walk for the ranks, parent from ranks.
 *   or_bfs          textbook FIFO BFS (Section III-A); parent = minimum-id
 *                   neighbour on the previous level.
 *   or_verify       exact RST verdict with a reason code.
 *   or_prrst        the PR-RST rounds of Section III-C simulated one step at a
 *                   time (alternating min/max hooking, path reversal);
 *                   or_prrst_from starts them from a given rooted forest
 *                   (edge insertions into an existing tree).
 *   or_bcc          biconnected components (blocks) and cut vertices by the
 *                   textbook depth-first search with an edge stack (Hopcroft
 *                   and Tarjan): the consumer of rooted trees that motivates
 *                   the paper (Section I).  Independent of any spanning tree.
 *
 * All CSR inputs use int64 offsets (the Python wrapper widens int32 ones),
 * int32 column ids and rows sorted ascending.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* verdict codes (the smallest failing code is reported) */
enum {
    ORV_VALID = 0,
    ORV_BAD_ROOT = 1,          /* root out of range or P[root] != root           */
    ORV_PARENT_RANGE = 2,      /* some P[v] outside [0, n)                         */
    ORV_NON_EDGE = 3,          /* some P[v] != v with (v, P[v]) not an arc of G    */
    ORV_CYCLE = 4,             /* some parent chain never reaches a self-parent    */
    ORV_NOT_SPANNING = 5,      /* an edge of G joins two different trees           */
    ORV_COMPONENT_ROOT = 6     /* a tree without r is not rooted at its min vertex */
};

/* ------------------------------------------------------------ union-find */

static int32_t uf_find(int32_t *p, int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }   /* path halving */
    return x;
}

/* --------------------------------------------------------------- Kruskal */

/*
 * Kruskal with union by rank.  Scanning rows u = 0..n-1 and, inside a row,
 * columns in the stored (ascending) order while keeping only v > u visits the
 * undirected edges exactly in ascending (min, max) key order; the row order is
 * checked first.  An edge is a tree edge iff it joins two different sets.
 *   label_out[v] = minimum vertex id of v's component
 *   tree_u/tree_v (capacity n) receive the tree edges, u < v, ascending key
 * Returns 0, or -1 for an id out of range, -2 for an unsorted row,
 * -3 for an allocation failure.
 */
int or_cc_kruskal(int64_t n, const int64_t *off, const int32_t *col,
                  int32_t *label_out, int32_t *tree_u, int32_t *tree_v,
                  int64_t *ntree_out) {
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t j = off[u]; j < off[u + 1]; ++j) {
            if (col[j] < 0 || col[j] >= n) return -1;
            if (j > off[u] && col[j] < col[j - 1]) return -2;
        }
    }
    int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    uint8_t *rk = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!p || !rk) { free(p); free(rk); return -3; }
    for (int64_t v = 0; v < n; ++v) p[v] = (int32_t)v;
    int64_t t = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t j = off[u]; j < off[u + 1]; ++j) {
            int32_t v = col[j];
            if (v <= u) continue;                 /* self-loop, or seen from row v */
            int32_t a = uf_find(p, (int32_t)u), b = uf_find(p, v);
            if (a == b) continue;
            if (rk[a] < rk[b]) { int32_t s = a; a = b; b = s; }
            p[b] = a;
            if (rk[a] == rk[b]) rk[a]++;
            tree_u[t] = (int32_t)u; tree_v[t] = v; ++t;
        }
    }
    /* label = min vertex id: the first vertex met per set in ascending order */
    int32_t *minv = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!minv) { free(p); free(rk); return -3; }
    for (int64_t v = 0; v < n; ++v) minv[v] = -1;
    for (int64_t v = 0; v < n; ++v) {
        int32_t r = uf_find(p, (int32_t)v);
        if (minv[r] < 0) minv[r] = (int32_t)v;
        label_out[v] = minv[r];
    }
    *ntree_out = t;
    free(minv); free(p); free(rk);
    return 0;
}

/* -------------------------------------------------- forest adjacency (CSR) */

typedef struct { int64_t *off; int32_t *adj; } adjlist;

static int build_adj(int64_t n, int64_t T, const int32_t *tu, const int32_t *tv, adjlist *g) {
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc((size_t)(2 * T + 1) * sizeof(int32_t));
    if (!g->off || !g->adj) return -3;
    for (int64_t k = 0; k < T; ++k) {
        if (tu[k] < 0 || tu[k] >= n || tv[k] < 0 || tv[k] >= n || tu[k] == tv[k]) return -1;
        g->off[tu[k] + 1]++; g->off[tv[k] + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    int64_t *cur = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!cur) return -3;
    for (int64_t v = 0; v < n; ++v) cur[v] = g->off[v];
    for (int64_t k = 0; k < T; ++k) {
        g->adj[cur[tu[k]]++] = tv[k];
        g->adj[cur[tv[k]]++] = tu[k];
    }
    free(cur);
    return 0;
}

/*
 * Parent array of the forest (tu, tv) of T edges on n vertices: the tree
 * holding `root` is rooted at root, every other tree at its minimum vertex id,
 * singletons point at themselves.  Iterative depth-first search.
 * Returns 0; -1 for a bad edge or root; -4 if the edge set has a cycle.
 */
int or_root_forest(int64_t n, int64_t T, const int32_t *tu, const int32_t *tv,
                   int32_t root, int32_t *parent_out) {
    if (n <= 0) return 0;
    if (root < 0 || root >= n) return -1;
    adjlist g;
    int rc = build_adj(n, T, tu, tv, &g);
    if (rc) { free(g.off); free(g.adj); return rc; }
    int32_t *stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int64_t visited_edges = 0;
    for (int64_t s = -1; s < n; ++s) {
        int32_t src = (s < 0) ? root : (int32_t)s;
        if (seen[src]) continue;
        int64_t sp = 0;
        stack[sp++] = src; seen[src] = 1; parent_out[src] = src;
        while (sp) {
            int32_t x = stack[--sp];
            for (int64_t j = g.off[x]; j < g.off[x + 1]; ++j) {
                int32_t y = g.adj[j];
                if (y == parent_out[x] && x != src) continue;
                if (seen[y]) { rc = -4; continue; }
                seen[y] = 1; parent_out[y] = x; stack[sp++] = y; ++visited_edges;
            }
        }
    }
    if (visited_edges != T) rc = -4;
    free(stack); free(seen); free(g.off); free(g.adj);
    return rc;
}

/* ---------------------------------------------------------- Euler tour */

typedef struct { int32_t src, dst; int64_t id; } oarc;

static int arc_cmp(const void *a, const void *b) {
    const oarc *x = (const oarc *)a, *y = (const oarc *)b;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    if (x->dst != y->dst) return x->dst < y->dst ? -1 : 1;
    return 0;
}

/*
 * Euler-tour rooting of Section III-D, one step after another.
 *   1. Arc k = (tu[k] -> tv[k]) and arc k+T = (tv[k] -> tu[k]) for k < T, so
 *      rev(e) = (e + E/2) mod E with E = 2T.
 *   2. Lexicographic sort of the arcs by (src, dst); first[v], last[v] are the
 *      first and last arc ids of v's run, next[e] the following arc of the run
 *      or -1.
 *   3. succ(e) = next(rev(e)) if that is not -1, else first(from(rev(e))).
 *   4. Tree roots: `root` for its tree, the minimum vertex id for the others;
 *      for every tree root r with arcs, succ(rev(last[r])) = -1.
 *   5. Ranks: walking succ from first[r] gives positions 0, 1, 2, ...
 *   6. Parent from ranks: for twins e = (u -> v), rev(e) = (v -> u), the twin
 *      with the smaller rank is traversed first and goes down the tree, so
 *      rank[e] < rank[rev(e)] gives parent[v] = u; otherwise parent[u] = v.
 *      (The printed rule states the case the other way round; this is the
 *      reading that yields P[root] = root and a valid tree.)
 * Outputs (all optional except parent_out):
 *   src_out/dst_out[i]: the i-th arc in sorted order (length 2T)
 *   rank_out[i]: rank of the i-th sorted arc
 * Returns 0, -1 for bad input, -3 allocation failure, -5 if a walk does not
 * cover its tree (the input was not a forest).
 */
int or_euler_tour(int64_t n, int64_t T, const int32_t *tu, const int32_t *tv, int32_t root,
                  int32_t *src_out, int32_t *dst_out, int32_t *rank_out, int32_t *parent_out) {
    if (n <= 0) return 0;
    if (root < 0 || root >= n) return -1;
    int64_t E = 2 * T;
    oarc *arcs = (oarc *)malloc((size_t)(E + 1) * sizeof(oarc));
    int64_t *from = (int64_t *)malloc((size_t)(E + 1) * sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc((size_t)(E + 1) * sizeof(int64_t));
    int64_t *first = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *last = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((size_t)(E + 1) * sizeof(int64_t));
    int64_t *succ = (int64_t *)malloc((size_t)(E + 1) * sizeof(int64_t));
    int64_t *rank = (int64_t *)malloc((size_t)(E + 1) * sizeof(int64_t));
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *troot = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int rc = 0;
    if (!arcs || !from || !pos || !first || !last || !next || !succ || !rank || !comp || !troot) {
        rc = -3; goto done;
    }
    /* 1. arcs */
    for (int64_t k = 0; k < T; ++k) {
        if (tu[k] < 0 || tu[k] >= n || tv[k] < 0 || tv[k] >= n || tu[k] == tv[k]) { rc = -1; goto done; }
        arcs[k].src = tu[k]; arcs[k].dst = tv[k]; arcs[k].id = k;
        arcs[k + T].src = tv[k]; arcs[k + T].dst = tu[k]; arcs[k + T].id = k + T;
    }
    for (int64_t e = 0; e < E; ++e) from[e] = arcs[e].src;
    /* 2. lexicographic sort, first/last/next (by arc id) */
    qsort(arcs, (size_t)E, sizeof(oarc), arc_cmp);
    for (int64_t v = 0; v < n; ++v) { first[v] = -1; last[v] = -1; }
    for (int64_t i = 0; i < E; ++i) {
        int64_t e = arcs[i].id;
        pos[e] = i;
        int32_t s = arcs[i].src;
        if (first[s] < 0) first[s] = e;
        last[s] = e;
        next[e] = (i + 1 < E && arcs[i + 1].src == s) ? arcs[i + 1].id : -1;
    }
    /* 3. succ */
    for (int64_t e = 0; e < E; ++e) {
        int64_t re = (e + T) % E;
        succ[e] = next[re] != -1 ? next[re] : first[from[re]];
    }
    /* 4. tree roots: components of the forest by union-find on its edges */
    for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)v;
    for (int64_t k = 0; k < T; ++k) {
        int32_t a = uf_find(comp, tu[k]), b = uf_find(comp, tv[k]);
        if (a == b) { rc = -5; goto done; }            /* a cycle: not a forest */
        if (a < b) comp[b] = a; else comp[a] = b;      /* set root = min vertex */
    }
    for (int64_t v = 0; v < n; ++v) troot[v] = uf_find(comp, (int32_t)v);  /* min vertex */
    {
        int32_t rc_root = troot[root];
        for (int64_t v = 0; v < n; ++v) if (troot[v] == rc_root) troot[v] = root;
    }
    for (int64_t v = 0; v < n; ++v) parent_out[v] = (int32_t)v;
    for (int64_t e = 0; e < E; ++e) rank[e] = -1;
    for (int64_t r = 0; r < n; ++r) {
        if (troot[r] != r || first[r] < 0) continue;
        int64_t tail = (last[r] + T) % E;             /* rev(last[r]) */
        succ[tail] = -1;
        /* 5. walk */
        int64_t e = first[r], k = 0;
        while (e != -1) {
            if (rank[e] != -1 || k >= E) { rc = -5; goto done; }
            rank[e] = k++;
            e = succ[e];
        }
    }
    for (int64_t e = 0; e < E; ++e) if (rank[e] < 0) { rc = -5; goto done; }
    /* 6. parent from ranks */
    for (int64_t k = 0; k < T; ++k) {
        if (rank[k] < rank[k + T]) parent_out[tv[k]] = tu[k];
        else parent_out[tu[k]] = tv[k];
    }
    for (int64_t i = 0; i < E; ++i) {
        if (src_out) src_out[i] = arcs[i].src;
        if (dst_out) dst_out[i] = arcs[i].dst;
        if (rank_out) rank_out[i] = (int32_t)rank[arcs[i].id];
    }
done:
    free(arcs); free(from); free(pos); free(first); free(last); free(next);
    free(succ); free(rank); free(comp); free(troot);
    return rc;
}

/* ------------------------------------------------------------------ BFS */

/*
 * Level-synchronous BFS expressed as a FIFO queue (Section III-A).  The
 * component of `root` is searched from root; every other component from its
 * minimum vertex id (the first unvisited id in ascending order).  Levels are
 * distances from the component's source.  parent[v] = the minimum-id
 * neighbour u with level[u] = level[v] - 1 (rows are sorted, so the first such
 * u in the row); sources point at themselves.
 * Returns 0, or -1 for a bad root / id.
 */
int or_bfs(int64_t n, const int64_t *off, const int32_t *col, int32_t root,
           int32_t *level_out, int32_t *parent_out) {
    if (n <= 0) return 0;
    if (root < 0 || root >= n) return -1;
    int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!q) return -3;
    for (int64_t v = 0; v < n; ++v) level_out[v] = -1;
    for (int64_t s = -1; s < n; ++s) {
        int32_t src = (s < 0) ? root : (int32_t)s;
        if (level_out[src] >= 0) continue;
        int64_t head = 0, tail = 0;
        q[tail++] = src; level_out[src] = 0;
        while (head < tail) {
            int32_t x = q[head++];
            for (int64_t j = off[x]; j < off[x + 1]; ++j) {
                int32_t y = col[j];
                if (y < 0 || y >= n) { free(q); return -1; }
                if (level_out[y] < 0) { level_out[y] = level_out[x] + 1; q[tail++] = y; }
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        parent_out[v] = (int32_t)v;
        if (level_out[v] == 0) continue;
        for (int64_t j = off[v]; j < off[v + 1]; ++j) {
            if (level_out[col[j]] == level_out[v] - 1) { parent_out[v] = col[j]; break; }
        }
    }
    free(q);
    return 0;
}

/* -------------------------------------------------------------- verifier */

static int has_arc(const int64_t *off, const int32_t *col, int32_t v, int32_t w) {
    int64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {                     /* binary search in the sorted row */
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < w) lo = mid + 1; else hi = mid;
    }
    return lo < off[v + 1] && col[lo] == w;
}

/*
 * Exact verdict for a parent array (codes above; the smallest failing code is
 * returned, each check running only when all smaller ones passed).
 * strict_roots: also require every tree without `root` to be rooted at its
 * minimum vertex id (code 6).
 */
int or_verify(int64_t n, const int64_t *off, const int32_t *col, int32_t root,
              const int32_t *parent, int strict_roots) {
    if (n <= 0) return ORV_VALID;
    if (root < 0 || root >= n || parent[root] != root) return ORV_BAD_ROOT;
    for (int64_t v = 0; v < n; ++v)
        if (parent[v] < 0 || parent[v] >= n) return ORV_PARENT_RANGE;
    for (int64_t v = 0; v < n; ++v)
        if (parent[v] != v && !has_arc(off, col, (int32_t)v, parent[v])) return ORV_NON_EDGE;
    /* every chain must reach a self-parent: walk with memoised tree roots */
    int32_t *tr = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *path = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *state = (uint8_t *)calloc((size_t)n, 1);   /* 0 new, 1 on path, 2 done */
    int verdict = ORV_VALID;
    for (int64_t v = 0; v < n && verdict == ORV_VALID; ++v) {
        if (state[v] == 2) continue;
        int64_t len = 0;
        int32_t x = (int32_t)v;
        while (state[x] == 0 && parent[x] != x) { state[x] = 1; path[len++] = x; x = parent[x]; }
        int32_t r;
        if (state[x] == 1) { verdict = ORV_CYCLE; break; }
        else if (state[x] == 2) r = tr[x];
        else { r = x; tr[x] = x; state[x] = 2; }
        for (int64_t k = 0; k < len; ++k) { tr[path[k]] = r; state[path[k]] = 2; }
    }
    if (verdict == ORV_VALID) {
        for (int64_t v = 0; v < n && verdict == ORV_VALID; ++v)
            for (int64_t j = off[v]; j < off[v + 1]; ++j)
                if (tr[col[j]] != tr[v]) { verdict = ORV_NOT_SPANNING; break; }
    }
    if (verdict == ORV_VALID && strict_roots) {
        /* tree root must be the min vertex of its tree (tree = component here) */
        int32_t *minv = path;
        for (int64_t v = 0; v < n; ++v) minv[v] = INT32_MAX;
        for (int64_t v = 0; v < n; ++v) if (v < minv[tr[v]]) minv[tr[v]] = (int32_t)v;
        int32_t rr = tr[root];
        for (int64_t v = 0; v < n; ++v)
            if (tr[v] == v && v != rr && minv[v] != v) { verdict = ORV_COMPONENT_ROOT; break; }
    }
    free(tr); free(path); free(state);
    return verdict;
}

/* ---------------------------------------------------------------- PR-RST */

/* rep[v] = root of v's tree in P, for all v, in O(n): walk up to the first
 * vertex whose root is known, then write the root along the walked path. */
static void tree_roots(int64_t n, const int32_t *P, int32_t *rep, int32_t *stack) {
    for (int64_t v = 0; v < n; ++v) rep[v] = -1;
    for (int64_t v = 0; v < n; ++v) {
        int64_t sp = 0;
        int32_t x = (int32_t)v;
        while (rep[x] < 0 && P[x] != x) { stack[sp++] = x; x = P[x]; }
        int32_t r = rep[x] >= 0 ? rep[x] : x;
        rep[x] = r;
        while (sp) rep[stack[--sp]] = r;
    }
}

/* Re-root the tree of P holding u at u and graft it under v (v == u: u just
 * becomes the root).  Path reversal (Section III-C): along the tree path
 * u = x0, x1 = P[x0], ..., xk = old root, every x_{i+1} takes x_i as parent;
 * the path is read from P (the state at the start of the round) and written
 * into Q. */
static void reverse_and_graft(const int32_t *P, int32_t *Q, int32_t u, int32_t v) {
    int32_t x = u;
    while (P[x] != x) { Q[P[x]] = x; x = P[x]; }
    Q[u] = v;
}

/*
 * PR-RST (Section III-C), simulated round by round.  Rooted forest P, every
 * vertex its own tree at the start.  Round t (t = 0, 1, ...) hooks with the
 * minimum rule when t is even and the maximum rule when t is odd: an arc
 * (u, v) whose trees have roots ru != rv is eligible for the tree ru when
 * rv < ru (minimum rule) or rv > ru (maximum rule), and each tree takes its
 * eligible arc with the smallest key (u, v).  A hooking tree is re-rooted at
 * u by path reversal and grafted under v.  The loop ends after the first
 * round without hooks.  Finally the tree of `root` is re-rooted at root and
 * every other tree at its minimum vertex id.
 *   rounds_out: number of rounds executed (the final hook-free one included)
 * Returns 0, -1 for a bad root or id.
 */
int or_prrst_from(int64_t n, const int64_t *off, const int32_t *col, int32_t root,
                  const int32_t *init, int32_t *parent_out, int64_t *rounds_out);

int or_prrst(int64_t n, const int64_t *off, const int32_t *col, int32_t root,
             int32_t *parent_out, int64_t *rounds_out) {
    return or_prrst_from(n, off, col, root, NULL, parent_out, rounds_out);
}

/*
 * The same rounds started from a given rooted forest instead of singletons:
 * the incremental use of PR-RST's graft and path reversal (Section III-C;
 * the paper's conclusion points to PR-RST for incremental graphs).  With
 * init a rooted spanning forest of G and (off, col) the arcs of G plus a
 * batch of new edges, only new edges can join two trees, so the result keeps
 * every tree edge of init (some reversed) and adds new edges only.
 *   init: n parents (roots P[r] = r), or NULL for singletons.
 */
int or_prrst_from(int64_t n, const int64_t *off, const int32_t *col, int32_t root,
                  const int32_t *init, int32_t *parent_out, int64_t *rounds_out) {
    if (n <= 0) { *rounds_out = 0; return 0; }
    if (root < 0 || root >= n) return -1;
    int32_t *P = parent_out;
    int32_t *Q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *rep = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *stk = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint64_t *best = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!Q || !rep || !best || !stk) { free(Q); free(rep); free(best); free(stk); return -3; }
    for (int64_t v = 0; v < n; ++v) {
        P[v] = init ? init[v] : (int32_t)v;
        if (P[v] < 0 || P[v] >= n) { free(Q); free(rep); free(best); free(stk); return -1; }
    }
    if (init) {  /* every parent chain must end at a root: rep[] = 0 unknown, 1 on the walk, 2 done */
        for (int64_t v = 0; v < n; ++v) rep[v] = 0;
        for (int64_t v = 0; v < n; ++v) {
            int64_t sp = 0;
            int32_t x = (int32_t)v;
            while (rep[x] == 0 && P[x] != x) { rep[x] = 1; stk[sp++] = x; x = P[x]; }
            if (rep[x] == 1) { free(Q); free(rep); free(best); free(stk); return -2; }  /* a cycle */
            rep[x] = 2;
            while (sp) rep[stk[--sp]] = 2;
        }
    }
    int64_t t = 0;
    for (;; ++t) {
        tree_roots(n, P, rep, stk);
        for (int64_t v = 0; v < n; ++v) best[v] = UINT64_MAX;
        for (int64_t u = 0; u < n; ++u) {
            for (int64_t j = off[u]; j < off[u + 1]; ++j) {
                int32_t v = col[j];
                if (v < 0 || v >= n) { free(Q); free(rep); free(best); free(stk); return -1; }
                int32_t ru = rep[u], rv = rep[v];
                if (ru == rv) continue;
                int eligible = (t % 2 == 0) ? (rv < ru) : (rv > ru);
                if (!eligible) continue;
                uint64_t key = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
                if (key < best[ru]) best[ru] = key;
            }
        }
        int any = 0;
        memcpy(Q, P, (size_t)n * sizeof(int32_t));
        for (int64_t r = 0; r < n; ++r) {
            if (rep[r] != r || best[r] == UINT64_MAX) continue;
            any = 1;
            reverse_and_graft(P, Q, (int32_t)(best[r] >> 32), (int32_t)(best[r] & 0xffffffffu));
        }
        memcpy(P, Q, (size_t)n * sizeof(int32_t));
        if (!any) break;
    }
    /* final re-rooting */
    tree_roots(n, P, rep, stk);
    int32_t *minv = (int32_t *)best;   /* reuse storage: n int32 fit in n uint64 */
    for (int64_t v = 0; v < n; ++v) minv[v] = INT32_MAX;
    for (int64_t v = 0; v < n; ++v) if (v < minv[rep[v]]) minv[rep[v]] = (int32_t)v;
    memcpy(Q, P, (size_t)n * sizeof(int32_t));
    for (int64_t r = 0; r < n; ++r) {
        if (rep[r] != r) continue;
        int32_t target = (r == rep[root]) ? root : minv[r];
        if (target != r) reverse_and_graft(P, Q, target, target);
    }
    memcpy(P, Q, (size_t)n * sizeof(int32_t));
    *rounds_out = t + 1;
    free(Q); free(rep); free(best); free(stk);
    return 0;
}

/* ------------------------------------------------------------ biconnected components */

/* First position of w in the sorted row v (every copy of a parallel edge is
 * named by its first copy), or -1. */
static int64_t first_pos(const int64_t *off, const int32_t *col, int32_t v, int32_t w) {
    int64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < w) lo = mid + 1; else hi = mid;
    }
    return (lo < off[v + 1] && col[lo] == w) ? lo : -1;
}

/*
 * Blocks of an undirected graph (maximal edge sets in which every two edges
 * lie on a common simple cycle; an edge on no cycle is a block by itself;
 * self-loops belong to no block).
 *   label[a]  (length A) for arc a = x->y: the smallest CSR position among
 *             the arcs of its block (the arc min->max of the block's
 *             lexicographically smallest edge); 0xFFFFFFFF for self-loops.
 *   cut[v]    1 iff v has edges in two or more blocks (a cut vertex).
 *   *nblocks  number of blocks.
 * Depth-first search from every unvisited vertex with discovery numbers and
 * low values; tree edges and back edges are pushed on an edge stack when
 * first met, and a block is popped when a child's low value does not reach
 * above its parent.  Parallel edges: only one copy of the edge to the parent
 * is skipped, the other copies are back edges.  Returns 0, or -1 on
 * allocation failure or asymmetric input.
 */
int or_bcc(int64_t n, const int64_t *off, const int32_t *col, uint32_t *label, uint8_t *cut,
           int64_t *nblocks) {
    const int64_t A = off[n];
    const size_t nn = (size_t)(n > 0 ? n : 1), aa = (size_t)(A > 0 ? A : 1);
    int64_t *disc = malloc(nn * sizeof(int64_t));
    int64_t *low = malloc(nn * sizeof(int64_t));
    int64_t *next = malloc(nn * sizeof(int64_t));     /* next arc of v to scan */
    int32_t *par = malloc(nn * sizeof(int32_t));      /* DFS parent (-1 at a start) */
    int64_t *in_arc = malloc(nn * sizeof(int64_t));   /* tree arc par->v */
    uint8_t *skipped = calloc(nn, 1);                 /* one copy of v->par skipped */
    int32_t *vst = malloc(nn * sizeof(int32_t));      /* vertex stack */
    int64_t *est = malloc(aa * sizeof(int64_t));      /* edge stack: arc positions */
    int32_t *esrc = malloc(aa * sizeof(int32_t));     /* and their sources */
    int64_t *blk = malloc(aa * sizeof(int64_t));      /* block of the edge named by first-copy min->max arc */
    int64_t *bmin = malloc(aa * sizeof(int64_t));     /* smallest position per block */
    int rc = 0;
    if (!disc || !low || !next || !par || !in_arc || !skipped || !vst || !est || !esrc || !blk || !bmin)
        rc = -1;
    for (int64_t v = 0; v < n && rc == 0; ++v) { disc[v] = -1; cut[v] = 0; }
    for (int64_t a = 0; a < A && rc == 0; ++a) blk[a] = -1;
    int64_t timer = 0, ne = 0, nb = 0;
    for (int64_t s = 0; s < n && rc == 0; ++s) {
        if (disc[s] >= 0) continue;
        int64_t top = 0;
        vst[top++] = (int32_t)s;
        disc[s] = low[s] = timer++;
        next[s] = off[s];
        par[s] = -1;
        in_arc[s] = -1;
        while (top > 0 && rc == 0) {
            const int32_t v = vst[top - 1];
            if (next[v] < off[v + 1]) {
                const int64_t a = next[v]++;
                const int32_t w = col[a];
                if (w == v) continue;                                   /* self-loop */
                if (w == par[v] && !skipped[v]) { skipped[v] = 1; continue; }  /* the entering edge */
                if (disc[w] < 0) {                                      /* tree edge */
                    est[ne] = a; esrc[ne] = v; ++ne;
                    disc[w] = low[w] = timer++;
                    next[w] = off[w];
                    par[w] = v;
                    in_arc[w] = a;
                    vst[top++] = w;
                } else if (disc[w] < disc[v]) {                         /* back edge to an ancestor */
                    est[ne] = a; esrc[ne] = v; ++ne;
                    if (disc[w] < low[v]) low[v] = disc[w];
                }                                                       /* else: met from w's side */
            } else {
                --top;
                const int32_t u = par[v];
                if (u < 0) continue;
                if (low[v] < low[u]) low[u] = low[v];
                if (low[v] >= disc[u]) {                                /* u separates v's subtree */
                    const int64_t id = nb++;
                    int64_t mn = INT64_MAX;
                    for (;;) {
                        if (ne <= 0) { rc = -1; break; }
                        --ne;
                        const int64_t e = est[ne];
                        const int32_t x = esrc[ne], y = col[e];
                        const int64_t p0 = first_pos(off, col, x < y ? x : y, x < y ? y : x);
                        if (p0 < 0) { rc = -1; break; }
                        blk[p0] = id;
                        if (p0 < mn) mn = p0;
                        if (e == in_arc[v]) break;
                    }
                    bmin[id] = mn;
                }
            }
        }
    }
    for (int64_t v = 0; v < n && rc == 0; ++v) {
        int64_t first = -1;
        for (int64_t a = off[v]; a < off[v + 1]; ++a) {
            const int32_t w = col[a];
            if (w == (int32_t)v) { label[a] = 0xFFFFFFFFu; continue; }
            const int64_t p0 = first_pos(off, col, (int32_t)v < w ? (int32_t)v : w, (int32_t)v < w ? w : (int32_t)v);
            if (p0 < 0 || blk[p0] < 0) { rc = -1; break; }
            const int64_t b = bmin[blk[p0]];
            label[a] = (uint32_t)b;
            if (first < 0) first = b;
            else if (b != first) cut[v] = 1;
        }
    }
    *nblocks = nb;
    free(disc); free(low); free(next); free(par); free(in_arc); free(skipped); free(vst);
    free(est); free(esrc); free(blk); free(bmin);
    return rc;
}
