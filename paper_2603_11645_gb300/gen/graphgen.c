/*
 * Seeded synthetic graph generators.
 *
 * This file builds the inputs that both the CUDA path and the CPU oracle
 * consume. It holds none of the spanning-tree method's arithmetic: it only
 * draws edges, permutes ids and packs an undirected edge list into a
 * symmetric CSR with sorted, duplicate-free rows and no self-loops.
 *
 * The workloads mirror the graph families of the paper's evaluation
 * (Section IV, Table II): high-diameter road/OSM-like graphs (grids, chains
 * with chords) and power-law graphs (R-MAT, Kronecker-like).
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based
 * stream so that every edge draw depends only on (seed, index).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ---- work splitting over threads ------------------------------------------
 * Every parallel loop below splits an index range into contiguous pieces and
 * writes disjoint outputs, so its result is the same for any thread count. */
typedef void (*gg_range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { gg_range_fn fn; void *ctx; int64_t lo, hi; } gg_piece;

static void *gg_piece_run(void *arg) {
    gg_piece *p = (gg_piece *)arg;
    p->fn(p->ctx, p->lo, p->hi);
    return NULL;
}

static int gg_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    const char *env = getenv("GG_THREADS");
    if (env && atoi(env) > 0) c = atoi(env);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

/* Runs fn over [0, k) in up to gg_threads() pieces (inline when small); a
 * piece whose thread cannot be started runs on the calling thread. */
static void gg_parallel(gg_range_fn fn, void *ctx, int64_t k) {
    int t = gg_threads();
    if (k < 65536 || t == 1) { fn(ctx, 0, k); return; }
    pthread_t th[64];
    gg_piece pc[64];
    int joined[64] = {0};
    for (int i = 0; i < t; ++i) {
        pc[i].fn = fn; pc[i].ctx = ctx;
        pc[i].lo = k * i / t; pc[i].hi = k * (i + 1) / t;
    }
    for (int i = 1; i < t; ++i)
        joined[i] = pthread_create(&th[i], NULL, gg_piece_run, &pc[i]) == 0;
    gg_piece_run(&pc[0]);
    for (int i = 1; i < t; ++i) {
        if (joined[i]) pthread_join(th[i], NULL);
        else gg_piece_run(&pc[i]);
    }
}

static inline uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t sm64_stream(uint64_t seed, uint64_t idx) {
    return seed * 0xd1b54a32d192ed03ULL + idx * 0xa0761d6478bd642fULL + 0x8bb84b93962eacc9ULL;
}

/* Uniform integer in [0, bound) by 128-bit multiply-shift (Lemire). */
static inline uint64_t sm64_below(uint64_t *x, uint64_t bound) {
    __uint128_t prod = (__uint128_t)sm64_next(x) * (__uint128_t)bound;
    return (uint64_t)(prod >> 64);
}

/* Fisher-Yates shuffle of the identity: out[i] is the new id of vertex i. */
void gg_permutation(int64_t n, uint64_t seed, int32_t *out) {
    uint64_t x = sm64_stream(seed, 0x5eed);
    for (int64_t i = 0; i < n; ++i) out[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&x, (uint64_t)(i + 1));
        int32_t t = out[i]; out[i] = out[j]; out[j] = t;
    }
}

/* Uniform draws in [0, bound) for k items, counter-based on (seed, i). */
void gg_uniform(int64_t k, uint64_t bound, uint64_t seed, int64_t *out) {
    for (int64_t i = 0; i < k; ++i) {
        uint64_t x = sm64_stream(seed, (uint64_t)i);
        out[i] = (int64_t)sm64_below(&x, bound);
    }
}

/*
 * R-MAT edge draws (Chakrabarti, Zhan, Faloutsos 2004): each of the m edges
 * descends `scale` levels of the adjacency matrix, choosing quadrant
 * (0,0),(0,1),(1,0),(1,1) with probability a,b,c,1-a-b-c. Each level uses
 * 32 bits of a SplitMix64 draw. Self-loops and duplicates are left in; the
 * CSR builder removes them.
 */
typedef struct {
    int scale;
    uint64_t ta, tab, tabc, seed;
    int32_t *u, *v;
} gg_rmat_ctx;

static void gg_rmat_range(void *c, int64_t lo, int64_t hi) {
    const gg_rmat_ctx *k = (const gg_rmat_ctx *)c;
    for (int64_t e = lo; e < hi; ++e) {
        uint64_t x = sm64_stream(k->seed, (uint64_t)e);
        uint32_t uu = 0, vv = 0;
        uint64_t bits = 0;
        for (int l = 0; l < k->scale; ++l) {
            if ((l & 1) == 0) bits = sm64_next(&x);
            uint64_t r = (l & 1) ? (bits >> 32) : (bits & 0xffffffffULL);
            uint32_t bu, bv;
            if (r < k->ta) { bu = 0; bv = 0; }
            else if (r < k->tab) { bu = 0; bv = 1; }
            else if (r < k->tabc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            uu = (uu << 1) | bu;
            vv = (vv << 1) | bv;
        }
        k->u[e] = (int32_t)uu;
        k->v[e] = (int32_t)vv;
    }
}

void gg_rmat_edges(int scale, int64_t m, double a, double b, double c,
                   uint64_t seed, int32_t *u, int32_t *v) {
    const double two32 = 4294967296.0;
    gg_rmat_ctx k;
    k.scale = scale;
    k.ta = (uint64_t)(a * two32);
    k.tab = (uint64_t)((a + b) * two32);
    k.tabc = (uint64_t)((a + b + c) * two32);
    k.seed = seed;
    k.u = u;
    k.v = v;
    gg_parallel(gg_rmat_range, &k, m);
}

/* ---- symmetric CSR construction --------------------------------------- */

static void isort_i32(int32_t *a, int64_t k) {
    for (int64_t i = 1; i < k; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

/* LSD radix sort of k non-negative int32 values using scratch tmp. */
static void rsort_i32(int32_t *a, int32_t *tmp, int64_t k) {
    int64_t cnt[256];
    int32_t *src = a, *dst = tmp;
    for (int shift = 0; shift < 32; shift += 8) {
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < k; ++i) cnt[((uint32_t)src[i] >> shift) & 255u]++;
        int64_t s = 0;
        for (int d = 0; d < 256; ++d) { int64_t t = cnt[d]; cnt[d] = s; s += t; }
        for (int64_t i = 0; i < k; ++i) dst[cnt[((uint32_t)src[i] >> shift) & 255u]++] = src[i];
        int32_t *t = src; src = dst; dst = t;
    }
    /* four passes: result is back in a */
}

typedef struct {
    int64_t n, m;
    const int32_t *u, *v;
    int64_t *cur;   /* per row: count (cols == NULL) or next free slot */
    int32_t *cols;  /* NULL: count only */
} gg_scatter_ctx;

static void gg_scatter_range(void *c, int64_t r0, int64_t r1) {
    const gg_scatter_ctx *k = (const gg_scatter_ctx *)c;
    for (int64_t e = 0; e < k->m; ++e) {
        int32_t a = k->u[e], b = k->v[e];
        if (a == b) continue;
        if (a >= r0 && a < r1) {
            if (k->cols) k->cols[k->cur[a]] = b;
            k->cur[a]++;
        }
        if (b >= r0 && b < r1) {
            if (k->cols) k->cols[k->cur[b]] = a;
            k->cur[b]++;
        }
    }
}

typedef struct {
    const int64_t *offsets;  /* row starts before compaction (offsets[i+1] = end of row i) */
    int32_t *cols;
    int64_t *deg;            /* out: row length after deduplication */
} gg_rows_ctx;

static void gg_rows_range(void *c, int64_t lo_row, int64_t hi_row) {
    const gg_rows_ctx *k = (const gg_rows_ctx *)c;
    int64_t cap = 0;
    int32_t *tmp = NULL;
    for (int64_t i = lo_row; i < hi_row; ++i) {
        int64_t lo = k->offsets[i], d = k->offsets[i + 1] - lo;
        int32_t *row = k->cols + lo;
        if (d <= 64) {
            isort_i32(row, d);
        } else {
            if (d > cap) {
                free(tmp);
                cap = d;
                tmp = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
            }
            rsort_i32(row, tmp, d);
        }
        int64_t w = 0;
        for (int64_t j = 0; j < d; ++j) {
            if (w > 0 && row[w - 1] == row[j]) continue;
            row[w++] = row[j];
        }
        k->deg[i] = w;
    }
    free(tmp);
}

/*
 * Build the symmetric CSR of an undirected edge list over vertices [0, n).
 * Self-loops are dropped; both arcs of every edge are stored; each row is
 * sorted ascending and duplicates are removed.
 *   offsets: n+1 entries (output)
 *   cols:    capacity 2*m (output, compacted in place)
 * Returns the number of stored arcs A = offsets[n], or -1 on a bad id.
 */
int64_t gg_build_csr(int64_t n, int64_t m, const int32_t *u, const int32_t *v,
                     int64_t *offsets, int32_t *cols) {
    for (int64_t e = 0; e < m; ++e)
        if (u[e] < 0 || v[e] < 0 || u[e] >= n || v[e] >= n) return -1;
    int64_t *cur = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cur) return -2;
    /* row lengths, then the arcs scattered into their rows; every thread owns
     * a range of rows and scans the whole edge list for them */
    gg_scatter_ctx sc = {n, m, u, v, cur, NULL};
    gg_parallel(gg_scatter_range, &sc, n);
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + cur[i];
    for (int64_t i = 0; i < n; ++i) cur[i] = offsets[i];
    sc.cols = cols;
    gg_parallel(gg_scatter_range, &sc, n);
    /* sort and deduplicate every row in place (rows in parallel), then
     * compact the rows to the front */
    int64_t *deg = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!deg) { free(cur); return -2; }
    gg_rows_ctx rc = {offsets, cols, deg};
    gg_parallel(gg_rows_range, &rc, n);
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo = offsets[i], d = deg[i];
        if (w != lo) memmove(cols + w, cols + lo, (size_t)d * sizeof(int32_t));
        offsets[i] = w;
        w += d;
    }
    offsets[n] = w;
    free(deg);
    free(cur);
    return w;
}

/* ---- connectivity patch for R-MAT --------------------------------------- */

static int32_t uf_find(int32_t *p, int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/*
 * Input recipe step for R-MAT inputs: for every connected component of the
 * edge list that does not contain vertex 0, emit one extra edge from the
 * component's minimum vertex id to vertex 0 (isolated vertices included).
 * Uses its own small union-find; this is input construction only.
 * Writes at most n-1 edges into out_u/out_v; returns the count.
 */
int64_t gg_connect_to_zero(int64_t n, int64_t m, const int32_t *u, const int32_t *v,
                           int32_t *out_u, int32_t *out_v) {
    int32_t *p = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!p) return -2;
    for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = uf_find(p, u[e]), b = uf_find(p, v[e]);
        if (a == b) continue;
        if (a < b) p[b] = a; else p[a] = b;   /* root = smaller id => root is the min vertex */
    }
    int32_t r0 = uf_find(p, 0);
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t r = uf_find(p, (int32_t)i);
        if (r == (int32_t)i && r != r0) { out_u[k] = (int32_t)i; out_v[k] = 0; ++k; }
    }
    free(p);
    return k;
}
