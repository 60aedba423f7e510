/*
 * rst.h -- C ABI of the GB300 rooted-spanning-tree library (librst.so).
 *
 * Method: "Beyond BFS: A Comparative Study of Rooted Spanning Tree Algorithms
 * on GPUs" (arXiv 2603.11645).  A rooted spanning tree (RST) of an undirected
 * graph G = (V, E) with root r is a parent array P with P[r] = r and exactly
 * one parent for every other vertex (Section I).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Graph input: symmetric CSR.  csr_offsets has n+1 entries, 32-bit or 64-bit
 *   as stated by offsets_bits (32 or 64); csr_cols has m = csr_offsets[n]
 *   entries (m counts DIRECTED arcs, i.e. twice the undirected edges).  Every
 *   undirected edge {u,v} is stored as both u->v and v->u, every row is sorted
 *   ascending, column ids are in [0, n).  Self-loops and repeated arcs are
 *   tolerated and never become tree edges.  Vertex ids are int32 and n must be
 *   below 2^30 (larger n returns RST_ERR_UNSUPPORTED: the up to 2(n-1) tree
 *   arcs of the Euler tour are indexed by int32); m must be below 2^32 (below 2^31 with
 *   32-bit offsets).
 * Memory: every array argument is caller-owned DEVICE memory unless marked
 *   "host".  The library never frees caller memory.  It keeps an internal
 *   per-device workspace that grows on demand (cudaMalloc) and is released by
 *   rst_shutdown().
 * Streams: work is issued on `stream` (a cudaStream_t; NULL = legacy default).
 *   In this version every entry point returns after its work has completed on
 *   that stream (it synchronises the stream), so outputs are ready on return.
 *   Calls are serialised per process; concurrent calls from several host
 *   threads are safe but do not overlap.
 * Disconnected inputs: the component of `root` is rooted at root; every other
 *   component is rooted at its minimum vertex id; isolated vertices point at
 *   themselves (the forest generalisation of Section III-D).
 * Errors: argument errors are detected before any GPU work and return
 *   RST_ERR_INVALID_ARG (or RST_ERR_UNSUPPORTED for sizes outside the limits
 *   above).  Errors detected by kernels (an index out of range in malformed
 *   input, a loop that exceeds its iteration bound) return RST_ERR_DEVICE or
 *   RST_ERR_NOT_CONVERGED; outputs are then unspecified.  CUDA API failures
 *   return RST_ERR_CUDA and allocation failures RST_ERR_OOM.
 */
#ifndef RST_H_
#define RST_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *rst_stream_t; /* identical to cudaStream_t */

typedef enum {
    RST_OK = 0,
    RST_ERR_INVALID_ARG = 1,
    RST_ERR_OOM = 2,
    RST_ERR_CUDA = 3,
    RST_ERR_NOT_CONVERGED = 4,
    RST_ERR_TIMEOUT = 5,
    RST_ERR_UNSUPPORTED = 6,
    RST_ERR_DEVICE = 7
} rst_status;

typedef enum {
    RST_AUTO = 0,      /* learned selector picks one of the three below        */
    RST_BFS = 1,       /* level-synchronous, direction-optimising BFS (III-A)  */
    RST_CC_EULER = 2,  /* hook/compress connectivity + Euler-tour rooting      */
    RST_PR_RST = 3,    /* path-reversal RST (III-C)                            */
    RST_CC_FAST = 4,   /* sampled union-find connectivity + Euler rooting      */
    RST_BFS_DEVICE = 5,     /* RST_BFS, level loop in a CUDA-graph while node  */
    RST_BFS_PERSISTENT = 6  /* RST_BFS, all levels in one cooperative launch   */
} rst_strategy;

/* Verdict codes written by rst_verify (the smallest failing code wins). */
enum {
    RST_VERDICT_VALID = 0,
    RST_VERDICT_BAD_ROOT = 1,       /* root out of range or P[root] != root         */
    RST_VERDICT_PARENT_RANGE = 2,   /* some P[v] outside [0, n)                      */
    RST_VERDICT_NON_EDGE = 3,       /* P[v] != v but (v, P[v]) is not an arc of G    */
    RST_VERDICT_CYCLE = 4,          /* a parent chain never reaches a self-parent    */
    RST_VERDICT_NOT_SPANNING = 5,   /* an edge of G joins two different trees        */
    RST_VERDICT_COMPONENT_ROOT = 6  /* a tree without root is not rooted at its min  */
};

/* Human-readable name of a status code (static storage). */
const char *rst_status_string(rst_status s);

/* Library version as 10000*major + 100*minor + patch. */
int rst_version(void);

/*
 * rst_build -- rooted spanning tree of a CSR graph (Section I, Section III).
 *   csr_offsets, offsets_bits, csr_cols, n, m: the graph (see conventions).
 *   root:       requested root, 0 <= root < n.
 *   strategy:   RST_CC_EULER (hook/compress connected components marking the
 *               tree edges, Section III-B, then Euler-tour rooting, Section
 *               III-D), RST_BFS (Section III-A), RST_PR_RST (Section III-C) or
 *               RST_AUTO (rst_select's choice).
 *   parent_out: n int32 (device), receives P.
 *               RST_BFS_DEVICE: the same search and result as RST_BFS with
               the level loop driven from the device (one kernel launch per
               level inside a CUDA-graph while loop, no host round trip per
               level): the stronger step-bound baseline.
               RST_BFS_PERSISTENT: the same search and result again, all
               levels inside one cooperative kernel launch whose blocks meet
               at a grid barrier after each level (bounded waits: a wait that
               runs out returns RST_ERR_NOT_CONVERGED).
               RST_CC_FAST: connectivity by sampled union-find hooking
 *               (Section III-B leaves the hooking rule open; this one links
 *               every vertex with its first two neighbours, then only the
 *               vertices outside the largest component with the rest of
 *               their rows, merging by compare-and-swap), then the same
 *               Euler-tour rooting.
 * CC+Euler, BFS and PR-RST results are unique and identical run to run:
 * CC+Euler roots the minimum spanning forest under edge keys (min(u,v),
 * max(u,v)); BFS takes for every vertex the minimum-id neighbour on the
 * previous level; PR-RST returns the forest its rounds build when every tree
 * grafts by its eligible edge of smallest (u, v) key (minimum rule first,
 * then alternating), re-rooted at the requested root.  RST_CC_FAST returns a
 * valid RST with the same components and tree roots, but its tree edges are
 * chosen by races (not reproducible run to run).
 */
rst_status rst_build(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols,
                     int64_t n, int64_t m, int32_t root, rst_strategy strategy,
                     int32_t *parent_out, rst_stream_t stream);

/*
 * rst_cc -- connected components and spanning-forest edges (Section III-B:
 * hooking marks each successful hook's edge as a spanning edge; pointer
 * jumping flattens the trees).
 *   labels_out:          n int32 (device, may be NULL); component id of each
 *                        vertex = the minimum vertex id of its component.
 *   tree_uv_out:         2*(n-1) int32 (device, may be NULL); tree edge t is
 *                        (tree_uv_out[2t], tree_uv_out[2t+1]) with u < v.  The
 *                        edge SET is the minimum spanning forest under keys
 *                        (min(u,v), max(u,v)); the ORDER of the list is
 *                        unspecified.
 *   num_tree_edges_out:  host int64 (may be NULL); receives T = n - #components.
 */
rst_status rst_cc(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols,
                  int64_t n, int64_t m, int32_t *labels_out, int32_t *tree_uv_out,
                  int64_t *num_tree_edges_out, rst_stream_t stream);

/*
 * rst_euler_root -- Euler-tour rooting of a forest (Section III-D).
 *   n:              number of vertices.
 *   tree_uv:        2*T int32 (device); edge t = (tree_uv[2t], tree_uv[2t+1]).
 *                   The edges must form a forest (no cycle, no repeated edge,
 *                   no self-loop); otherwise RST_ERR_DEVICE.
 *   num_tree_edges: T (0 <= T < n).
 *   root:           requested root.
 *   parent_out:     n int32 (device), receives P.
 *   rank_out:       2*T int32 (device, may be NULL).  Position of each arc in
 *                   its tree's tour (0 = the root's first arc), indexed by the
 *                   arc's place in lexicographic (src, dst) order.  The tour
 *                   follows succ(e) = next(rev(e)), or first(from(rev(e))) at
 *                   the end of a run, and each tree's cycle is broken at
 *                   rev(last[tree root]).
 */
rst_status rst_euler_root(int64_t n, const int32_t *tree_uv, int64_t num_tree_edges,
                          int32_t root, int32_t *parent_out, int32_t *rank_out,
                          rst_stream_t stream);

/*
 * rst_build_batch -- rooted spanning trees of many independent graphs in one
 * call.  The batch is processed as one disjoint union, so fixed per-call and
 * per-launch costs are paid once per batch instead of once per graph (the
 * launch cost is what the paper blames for BFS's slowness, Section IV-B).
 *   Layout (all device memory):
 *     packed_offsets: the graphs' CSR offset arrays concatenated; graph g's
 *                     n_g + 1 LOCAL offsets (starting at 0) begin at index
 *                     graph_vtx_off[g] + g; 32- or 64-bit (offsets_bits).
 *     packed_cols:    the graphs' column arrays concatenated, LOCAL ids.
 *     graph_vtx_off, graph_arc_off: num_graphs + 1 int64 each; prefix sums of
 *                     the graphs' vertex and arc counts.
 *     roots:          num_graphs int32, local root of each graph.
 *     parent_out:     graph_vtx_off[num_graphs] int32; parent_out[
 *                     graph_vtx_off[g] + v] = LOCAL parent of v in graph g.
 *   strategy: RST_CC_EULER (RST_AUTO maps to it) or RST_BFS (one
 *   multi-source search from all roots); RST_PR_RST returns
 *   RST_ERR_UNSUPPORTED.  Each graph's result equals rst_build on that graph.
 */
rst_status rst_build_batch(const void *packed_offsets, int offsets_bits, const int32_t *packed_cols,
                           const int64_t *graph_vtx_off, const int64_t *graph_arc_off,
                           int32_t num_graphs, const int32_t *roots, rst_strategy strategy,
                           int32_t *parent_out, rst_stream_t stream);

/*
 * rst_verify -- exact validity check of a parent array (the RST definition of
 * Section I, extended to forests as in Section III-D).
 *   parent:      n int32 (device).
 *   verdict_out: host int32; one of RST_VERDICT_*.  The check for code k runs
 *                only when all codes below k passed, so the smallest failing
 *                code is reported.
 */
rst_status rst_verify(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols,
                      int64_t n, int64_t m, int32_t root, const int32_t *parent,
                      int32_t *verdict_out, rst_stream_t stream);

/* rst_bcc -- blocks (biconnected components) and cut vertices, computed from
 * the CC+Euler rooted spanning forest the way Tarjan and Vishkin do: subtree
 * intervals from the Euler-tour ranks, low/high values by range queries, and
 * connectivity of the auxiliary graph on tree edges (the downstream use of
 * rooted spanning trees named in Section I).
 *   csr_offsets, offsets_bits, csr_cols, n, m: the graph (see conventions).
 *   block_out       device uint32[m]: for arc a = x->y, the smallest CSR
 *                   position among the arcs of the block holding edge {x, y}
 *                   (so two arcs share a block iff their values are equal;
 *                   the value does not depend on any spanning tree);
 *                   0xFFFFFFFF for a self-loop, which lies in no block.
 *   cut_out         device uint8[n] or NULL: 1 iff the vertex has edges in two
 *                   or more blocks.
 *   num_blocks_out  host int64 or NULL: number of blocks.
 * A block is a maximal set of edges any two of which lie on a common simple
 * cycle; an edge on no cycle (a bridge) is a block by itself; parallel edges
 * form a cycle.  Workspace: about 130 bytes per vertex beyond rst_build's
 * (the range tables over the tour take 80). */
rst_status rst_bcc(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols, int64_t n, int64_t m,
                   uint32_t *block_out, uint8_t *cut_out, int64_t *num_blocks_out, rst_stream_t stream);

/* rst_insert_edges -- update a rooted spanning forest after inserting edges,
 * with PR-RST's graft and path reversal (Section III-C; the paper's
 * conclusion names PR-RST as the path for incremental graphs).
 *   n       number of vertices (unchanged by the insertion).
 *   parent  device int32[n], in and out.  In: a rooted spanning forest of
 *           the current graph G (parent[r] == r exactly at roots).  Out: a
 *           rooted spanning forest of G plus the new edges: every old tree
 *           edge is kept (some reoriented), only new edges are added; the tree
 *           holding `root` is rooted at root, every other tree at its minimum
 *           vertex.
 *   new_uv  device int32[2k]: the inserted undirected edges {new_uv[2i],
 *           new_uv[2i+1]} (self-loops and edges inside one tree change
 *           nothing).
 * The PR-RST rounds run from the given forest over the new edges only
 * (minimum rule, then maximum, alternating; each tree takes its eligible
 * edge with the smallest (u, v) key), which gives the same result as PR-RST
 * rounds over all edges of the new graph started from that forest.
 *   flags   0, or RST_INSERT_CANONICAL: the caller declares that the input
 *           is already in this canonical form for `root` (the tree holding
 *           root rooted at root, every other tree at its minimum vertex), as
 *           rst_build and rst_insert_edges return it.  Then only the trees the
 *           batch merges are re-rooted at the end (work proportional to the
 *           batch when their paths are short); for any other input the
 *           output is unspecified.  Without the flag every tree is re-rooted,
 *           whatever the input.
 * Batches of at most n/64 edges run their rounds sparsely: each end walks to
 * its root (at most the "insert_walk_limit" option's steps; a longer walk
 * hands the rounds to the dense version, over all vertices, at the same
 * round, with the same result).
 * Returns RST_ERR_DEVICE for an id outside [0, n), RST_ERR_INVALID_ARG for an
 * unknown flag and RST_ERR_NOT_CONVERGED when `parent` holds a cycle. */
enum { RST_INSERT_CANONICAL = 1 };
rst_status rst_insert_edges(int64_t n, int32_t *parent, const int32_t *new_uv, int64_t k, int32_t root,
                            unsigned int flags, rst_stream_t stream);

/* rst_tree_depth -- depth of every vertex of a rooted forest, and its height
 * (Section IV-B, Fig. 2: the trees of connectivity-based strategies are
 * deeper than BFS trees; this measures that trade-off on any parent array).
 *   parent     device int32[n], parent[v] == v exactly at roots (the output of
 *              rst_build with any strategy).
 *   depth_out  device int32[n] or NULL: edges from v up to its root.  Used as
 *              scratch during the call.
 *   max_out    host int64 or NULL: the largest depth (0 for an edgeless forest).
 * Pointer jumping with distances, about log2(height) + 1 rounds.  Returns
 * RST_ERR_INVALID_ARG for a parent outside [0, n) and RST_ERR_NOT_CONVERGED
 * when some parent chain never reaches a root (a cycle).  Synchronises
 * `stream` once per round. */
rst_status rst_tree_depth(const int32_t *parent, int64_t n, int32_t *depth_out, int64_t *max_out,
                          rst_stream_t stream);

/*
 * rst_build_noalloc -- the CC+Euler rooted spanning tree of rst_build, for
 * callers that cannot allocate device memory.  Such callers include a
 * serving process or an embedding runtime that reserves its whole device
 * memory budget at start-up (a pool that the library cannot draw from), and
 * hosts whose allocator must not be entered from the calling thread.  The
 * paper has no counterpart; this is a deployment variant of the same
 * computation, with the same result.
 *   Arguments and output are those of rst_build with RST_CC_EULER; the
 *   caller still provides the graph and parent_out in device memory.
 *   Limits: n <= 65,536 vertices and m <= 524,288 arcs; larger inputs return
 *   RST_ERR_UNSUPPORTED before any GPU work.
 *   Memory: it never calls cudaMalloc, cudaFree, cudaMallocHost or any other
 *   allocating routine (nor creates events, streams or graphs).  Its
 *   workspace is a 16 MiB array defined inside the library that every GPU
 *   loading the library holds until process exit.
 *   Set-up: the first call on a device looks up that array's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture begins.
 *   Like every entry point it returns after its work has completed on
 *   `stream`: it reads the round count and its status word back between
 *   rounds and at the end.
 *   Sharing: every call on a device uses the same array, which keeps the
 *   previous call's contents (the call clears what must start at zero).
 *   Calls whose GPU work overlaps (different streams without ordering) race
 *   on the array; host-side calls are serialised.
 */
rst_status rst_build_noalloc(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols,
                             int64_t n, int64_t m, int32_t root, int32_t *parent_out,
                             rst_stream_t stream);

/* ---- learned strategy selector (no counterpart in the paper) ---------------
 * The paper's comparison (Section IV) shows that the fastest strategy depends
 * on the graph's depth.  The selector maps 12 cheap features to predicted
 * natural-log times of BFS, CC+Euler and PR-RST with a 12-64-64-3 ReLU MLP and
 * picks the smallest, falling back to CC+Euler when the predicted advantage of
 * another strategy is below a margin.
 *
 * rst_selector_features: writes the 12 features (host float[12]) of a graph,
 *   computed on the device: log2 n, log2 m, mean degree, degree CV, degree
 *   skewness, log2(1+max deg), fraction of degree <= 2, log2(1+vertices
 *   reached by an 8-level BFS probe from root), log2 frontier growth between
 *   probe levels 3 and 7, log2 of an eccentricity estimate, log2(round-1 hook
 *   components / n), and the fraction of the m edges that survive one hook
 *   pass (edges u < v whose ends lie in different round-1 components of the
 *   min-key hooking of Section III-B).
 * rst_selector_load: installs network parameters (host float[5187]: W1[64][12],
 *   b1[64], W2[64][64], b2[64], W3[3][64], b3[3]), normalisation (host
 *   float[30]: feature means[12], feature stds[12], target means[3], target
 *   stds[3]) and the fallback margin (in log-time units).
 * rst_select: features, prediction and choice, all on the device; choice_out
 *   (host) and pred_log_time_out (host float[3], may be NULL).  Without loaded
 *   parameters it chooses RST_CC_EULER.  rst_build with RST_AUTO uses the
 *   same choice.
 * rst_selector_predict: the loaded network applied on the device to `batch`
 *   feature rows (device float[batch][12], raw as rst_selector_features
 *   writes them): pred_out (device float[batch][3] or NULL) receives the
 *   predicted natural-log times (BFS, CC+Euler, PR-RST), choice_out (device
 *   int32[batch] or NULL) the rst_strategy rst_select would pick.
 *   RST_ERR_UNSUPPORTED when no parameters are loaded.
 * rst_mlp_forward / rst_mlp_loss_grad / rst_mlp_adam / rst_mlp_train: the
 *   network's FP32 forward pass, mean-squared-error loss and gradient, Adam
 *   step (Kingma & Ba) and a full-batch training loop, all on device arrays
 *   (params[5187], X[batch][12] standardised, T[batch][3], grad[5187],
 *   adam_m/adam_v[5187], loss_out float[1], loss_hist float[epochs]).
 * rst_set_option: "bfs_max_levels" caps BFS at that many levels (0: no cap;
 *   a capped search returns RST_ERR_NOT_CONVERGED) -- used to censor BFS
 *   timings on very deep graphs when collecting selector training data.
 *   The other keys change speed only, never a result.  They play the part of
 *   the launch-granularity choice Section III-C makes for PR-RST (several
 *   pointer jumps per global synchronisation, chosen empirically); the
 *   package's autotune module searches them offline per size bucket:
 *     "lr_spacing"            list-ranking splitter spacing K of the first
 *                             level, a power of two in [16, 512] (default 16;
 *                             the deeper, L2-resident levels use 8);
 *     "round_blocks_per_sm"   grid of the contraction-round kernels, in resident
 *                             256-thread blocks per SM, [1, 16] (default 8;
 *                             the hook and resolve kernels take at most 6 and
 *                             5, the blocks their registers let reside);
 *     "bfs_bottom_up_divisor" BFS steps bottom-up while the frontier holds more
 *                             than n / divisor vertices, [1, 10^6] (default 20);
 *     "bfs_device_blocks_per_sm"     grid of RST_BFS_DEVICE's level kernel in
 *                             256-thread blocks per SM, [1, 8] (default 2);
 *     "bfs_persistent_blocks_per_sm" grid of RST_BFS_PERSISTENT, at most this
 *                             many resident blocks per SM, [1, 8] (default 1);
 *     "insert_walk_limit"     rst_insert_edges runs its rounds sparsely (work
 *                             proportional to the batch: walks from the new
 *                             edges' ends to their roots, per-tree path
 *                             reversal) while batches have at most n/64 edges
 *                             and every walk stays within this many steps,
 *                             otherwise over all vertices; [0, 2^30], 0 =
 *                             never sparse (default 2048);
 *     "euler_block"           threads per block of the Euler stage's
 *                             grid-stride kernels (run boundaries, successors,
 *                             parents from ranks): 128, 256 or 512 (default
 *                             256);
 *     "pr_levels_per_launch"  PR-RST computes this many pointer-jumping
 *                             levels per launch and host check, [1, 3]
 *                             (default 1; each level is recomputed exactly);
 *     "giant_share_pct"       CC+Euler: when one round-1 component holds at
 *                             least this percentage of a fixed sample of the
 *                             vertices with edges, the contracted edge list is
 *                             built from the rows of the other vertices only
 *                             (the giant's rows are not read); [0, 101]
 *                             (default 75; 0 = always from the largest
 *                             sampled component, 101 = never).
 *   Out-of-range values and unknown keys return RST_ERR_INVALID_ARG and change
 *   nothing.  Options are process-wide: set them between calls, not during.
 * rst_get_option: reads the current value of any key above into *value (host). */
rst_status rst_selector_features(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols,
                                 int64_t n, int64_t m, int32_t root, float *features_out,
                                 rst_stream_t stream);
rst_status rst_selector_load(const float *params, const float *norm, float margin);
rst_status rst_select(const void *csr_offsets, int offsets_bits, const int32_t *csr_cols, int64_t n,
                      int64_t m, int32_t root, rst_strategy *choice_out, float *pred_log_time_out,
                      rst_stream_t stream);
rst_status rst_selector_predict(const float *features, int batch, float *pred_out, int32_t *choice_out,
                                rst_stream_t stream);
rst_status rst_mlp_forward(const float *params, const float *X, int batch, float *Y,
                           rst_stream_t stream);
rst_status rst_mlp_loss_grad(const float *params, const float *X, const float *T, int batch,
                             float *grad, float *loss_out, rst_stream_t stream);
rst_status rst_mlp_adam(float *params, const float *grad, float *m, float *v, int count, int step,
                        float lr, float beta1, float beta2, float eps, rst_stream_t stream);
rst_status rst_mlp_train(float *params, const float *X, const float *T, int batch, int epochs,
                         float lr, float *adam_m, float *adam_v, float *loss_hist,
                         rst_stream_t stream);
rst_status rst_set_option(const char *key, long long value);
rst_status rst_get_option(const char *key, long long *value);

/* ---- diagnostics (no counterpart in the paper) ----------------------------
 * rst_launch_count: number of kernels this library has launched since load.
 * rst_profile_enable(1) starts recording a CUDA event at each stage boundary
 * of subsequent calls (on the call's stream); rst_profile_read writes up to
 * max_stages stage durations in milliseconds and their static names (host
 * arrays, may be NULL), returns the count and clears the record.
 * rst_profile_enable(0) stops recording. */
long long rst_launch_count(void);
/* Sizes seen by the last call (host array): hooking rounds, components with
 * edges after round 1, inter-component edges after round 1, tree edges,
 * components with edges, BFS levels or list-ranking levels, tree arcs list-
 * ranked (after leaf pruning), and for CC+Euler the hooking rounds finished
 * by one thread block once few components remain (0: none) and the times
 * that block handed back to the grid-wide rounds because the remaining
 * component pairs did not fit, and the number of vertices whose rows built
 * the contracted edge list when a giant round-1 component was found (-1:
 * every row was read).  Returns the number of values written (at most max,
 * at most 10). */
int rst_last_stats(long long *out, int max);
void rst_profile_enable(int on);
/* Record only the stage marks named in `names` (comma-separated, as returned
 * by rst_profile_read; NULL or "" records every mark).  A recorded mark is an
 * event between two kernels, which also keeps the second from being
 * scheduled while the first drains; timing a few stages this way leaves the
 * rest of the call as it runs unprofiled. */
void rst_profile_only(const char *names);
int rst_profile_read(float *ms_out, const char **names_out, int max_stages);

/* Release the internal workspace of every device the library touched. */
rst_status rst_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* RST_H_ */
