// Internal interfaces between the pipeline stages (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace rst {

constexpr uint32_t kNone = 0xffffffffu;

// Rank of bit j in a bitmap (e.g. CSR position j among the tree arcs): the
// number of set bits before j.  wpre[w] = popcount of words [0, w).
__device__ __forceinline__ uint32_t bit_rank(const uint32_t* __restrict__ bits,
                                             const uint32_t* __restrict__ wpre, uint64_t j) {
  uint64_t w = j >> 5;
  uint32_t lowmask = (1u << (uint32_t)(j & 31)) - 1u;
  return wpre[w] + (uint32_t)__popc(bits[w] & lowmask);
}
// The same from the interleaved {word, prefix} array of scan_popcount_ranked:
// one 8-byte read instead of two 4-byte ones.
__device__ __forceinline__ uint32_t bit_rank2(const uint2* __restrict__ rk, uint64_t j) {
  const uint2 e = rk[j >> 5];
  return e.y + (uint32_t)__popc(e.x & ((1u << (uint32_t)(j & 31)) - 1u));
}

// ----------------------------------------------------------------- CC
// Output of the hook/compress connectivity pass (Section III-B).
struct CcOut {
  int64_t T = 0;             // number of tree edges (= n - #components)
  uint4* pairs = nullptr;    // T records {p, q, a, b}: tree edge {a,b}; p = CSR
                             // position of arc a->b (row a), q of b->a (row b)
  uint32_t* bits = nullptr;  // bitmap over CSR positions: both arcs of every tree edge
  int64_t nroots = 0;        // number of components with at least one edge
  int32_t* roots = nullptr;  // their minimum vertex ids (canonical labels)
  int rounds = 0;            // hooking rounds executed (round 1 included)
  int32_t root_label = -1;   // canonical label of the requested root (host value)
  // Several requested roots (disjoint-union batches): rootof[L] is the root
  // requested for the component whose canonical label is L, or -1.  When set
  // it replaces root / root_label.
  const int32_t* rootof = nullptr;
  // Set when the connectivity pass already started the Euler stage's first
  // steps while the host read its counts back: the ranked tree-arc bitmap
  // (A/32 + 2 {word, prefix} pairs, from bits), a zeroed root bitmap
  // (n/32 + 1 words) and the row-start bitmap (row_starts below).
  uint2* rk = nullptr;
  unsigned long long* rk_tmp = nullptr;  // the scan's scratch (reused by later scans)
  uint32_t* root_bits = nullptr;
  uint32_t* rs = nullptr;
};

// Row-start bitmap over CSR positions (A/32 + 2 words): bit j is set when a
// non-empty row starts at position j, and bit A closes the last row.  With
// the tree-arc bitmap it tells, for a tree arc, whether another tree arc
// follows it in its row and where its row starts, from two small
// L2-resident bitmaps instead of the vertex's offsets.
int64_t row_start_words(int64_t A);
// The bit of vertex v (v <= n; o = off[v], o1 = off[v+1] for v < n), called
// by every lane of a warp for consecutive v (lanes past n pass v > n).
// Offsets are non-decreasing, so a warp's positions fall in a few
// consecutive words: the bits of one word are OR-ed across the warp first (a
// segmented suffix OR by shuffles) and its first lane sets them with one
// atomic.  rs must start zeroed.
template <class OffT>
__device__ __forceinline__ void row_start_bit(uint32_t* __restrict__ rs, const OffT*, int64_t n, int64_t v,
                                              uint64_t o, uint64_t o1) {
  const int lane = threadIdx.x & 31;
  int64_t word = -1;  // lanes past n belong to no word
  uint32_t bit = 0;
  if (v <= n) {
    word = (int64_t)(o >> 5);
    if (v == n || o1 > o) bit = 1u << (o & 31);  // v == n: the end of the last row
  }
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t b2 = __shfl_down_sync(0xffffffffu, bit, d);
    const int64_t w2 = __shfl_down_sync(0xffffffffu, word, d);
    if (lane + d < 32 && w2 == word) bit |= b2;
  }
  const int64_t wprev = __shfl_up_sync(0xffffffffu, word, 1);
  if (word >= 0 && bit && (lane == 0 || wprev != word)) atomicOr(&rs[word], bit);
}
template <class OffT>
rst_status row_starts(const OffT* off, int64_t n, int64_t A, uint32_t* rs, cudaStream_t s);

struct CcPlan;  // workspace layout, defined in cc.cu

// Connected components + spanning forest.  `labels_out` (nullable) receives the
// canonical label of every vertex.  `root` (may be -1) selects the vertex whose
// component label is returned in out->root_label.  With prefetch_euler the
// Euler stage's bitmap scan and root-flag clear are queued behind the count
// read-back, so the GPU runs them while the host waits (out->rk, out->root_bits,
// out->rs).
template <class OffT>
rst_status cc_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A,
                  int32_t root, int32_t* labels_out, CcOut* out, cudaStream_t s,
                  bool prefetch_euler = false);
template <class OffT>
size_t cc_workspace_bytes(int64_t n, int64_t A);
// Release cached round graphs (rst_shutdown).
void destroy_round_graphs();
// Round 1 of the hooking alone (cc.cu): P = round-1 roots, tree-edge records
// counted in counters[0], their arcs marked in bits.
template <class OffT>
rst_status round1_forest(const OffT* off, const int32_t* col, int64_t n, int32_t* P, uint32_t* J,
                         uint4* pairs, uint32_t* bits, unsigned long long* counters, cudaStream_t s);
// The same outputs from sampled union-find hooking (ccfast.cu): a valid
// spanning forest with the same components, chosen by races (not unique).
template <class OffT>
rst_status ccfast_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A,
                      int32_t root, int32_t* labels_out, CcOut* out, cudaStream_t s);
template <class OffT>
size_t ccfast_workspace_bytes(int64_t n, int64_t A);

// ----------------------------------------------------------------- Euler

// CSR-bitmap front end: converts CC output into tree positions, marks roots
// (the requested root for its component, the minimum vertex otherwise), sets
// P[v] = v for roots and singletons, builds the Euler successors, ranks the
// tours and sets every other parent from the ranks.
template <class OffT>
rst_status euler_root_cc(Arena& ar, const OffT* off, int64_t n, int64_t A, int32_t root,
                         CcOut* cc, int32_t* parent_out, uint32_t* rank_out, cudaStream_t s,
                         const int32_t** succ_view = nullptr);
size_t euler_cc_workspace_bytes(int64_t n, int64_t A, int64_t T, int64_t nroots);

// Edge-list front end (rst_euler_root): radix-sorts the 2T arcs by (src, dst).
rst_status euler_root_edges(Arena& ar, int64_t n, const int32_t* tree_uv, int64_t T, int32_t root,
                            int32_t* parent_out, uint32_t* rank_out, cudaStream_t s);
size_t euler_edges_workspace_bytes(int64_t n, int64_t T);

// ----------------------------------------------------------------- list ranking
// pos[x] = sum of weights of the elements before x in its list (weights 1 when
// w == nullptr).  nxt[x] = successor or -1.  heads: one entry per list.
//
// With `first` set, the first level's final pass may be left out: its records
// are then described in *first (valid = true) and pos is NOT written; the
// caller derives any element's position with lr_position().
struct LrFirstLevel {
  bool valid = false;
  const int2* ol = nullptr;        // {owner splitter, offset} (overflow and unpacked records)
  const uint32_t* ol32 = nullptr;  // packed records (owner << fbits | offset), or null
  int fbits = 0;
  const uint32_t* spos = nullptr;  // positions of the splitters
  int64_t S = 0;                   // number of splitters
  const unsigned long long* visited = nullptr;  // elements the walks reached (must be N)
  int64_t N = 0;
};
rst_status list_rank(Arena& ar, int64_t N, const int32_t* nxt, const uint32_t* w,
                     const int32_t* heads, int64_t nheads, uint32_t* pos, cudaStream_t s,
                     LrFirstLevel* first = nullptr);
// Position of element x from first-level records (kNone for an element no walk
// reached, whose record holds stale data: its owner is bounds-checked).
__device__ __forceinline__ uint32_t lr_position(const int2* __restrict__ ol, const uint32_t* __restrict__ ol32,
                                                int fbits, const uint32_t* __restrict__ spos, int64_t S,
                                                uint32_t x) {
  int2 r;
  if (ol32) {
    const uint32_t v = ol32[x];
    r = v != 0xffffffffu ? make_int2((int32_t)(v >> fbits), (int32_t)(v & ((1u << fbits) - 1u))) : ol[x];
  } else {
    r = ol[x];
  }
  return (r.x >= 0 && (int64_t)r.x < S) ? spos[r.x] + (uint32_t)r.y : kNone;
}
size_t list_rank_workspace_bytes(int64_t N, int64_t nheads);
// Upper bound over any number of heads.
size_t list_rank_workspace_upper(int64_t N);

// ----------------------------------------------------------------- sort
// Stable LSD radix sort of 64-bit keys on their low `key_bits` bits.
size_t radix_sort_workspace_bytes(int64_t count);
rst_status radix_sort_keys(Arena& ar, uint64_t* keys, int64_t count, int key_bits, cudaStream_t s);

}  // namespace rst
