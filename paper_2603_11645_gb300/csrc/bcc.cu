// Biconnected components (blocks) and cut vertices on top of the Euler tour:
// the consumer of rooted spanning trees that motivates the paper (Section I),
// computed the Tarjan-Vishkin way from a rooted spanning forest.
//
//  1 spanning forest + Euler-tour ranks (the CC+Euler path, root 0, no leaf
//    pruning).  The tours of the trees are laid end to end (tree j's arcs at
//    global positions base_j .. base_j + len_j - 1), so a non-root vertex x
//    owns the interval [key(x), end(x)] = positions of its down arc and of its
//    up arc, and y lies in x's subtree iff key(x) <= key(y) <= end(x).  A tree
//    root gets key = base_j - 1 and end = base_j + len_j - 1.
//  2 local values: lo(x) = min(key(x), key(y) over non-tree edges {x, y}),
//    hi(x) the max.  Numbering the non-root vertices by the order of their
//    down arcs (the preorder; a popcount rank over a bitmap of down-arc
//    positions) makes x's subtree the index range [idx(x), idx(x) + nd(x) - 1],
//    nd(x) = (end(x) - key(x) + 1) / 2, so low(x) / high(x) are range-min/max
//    queries over {lo, hi} pairs stored at idx: a sparse table inside every
//    32-index block (built with warp shuffles) plus one over block extremes.
//  3 the auxiliary graph on tree edges (tree edge p(w)-w named by w):
//      a non-tree edge {x, y} between unrelated vertices joins x and y;
//      a tree edge u-w with u not a root joins w and u when
//      low(w) < key(u) or high(w) > end(u) (w's subtree reaches outside u's);
//    its components (union-find, CAS hooking) are the blocks.  A non-tree
//    edge belongs to the block of its endpoint with the larger key.
//  4 labels: every arc gets the smallest CSR position among its block's arcs
//    (unique, independent of the spanning tree); a vertex whose arcs carry two
//    or more labels is a cut vertex.
#include <climits>

#include "csr_walk.cuh"
#include "pipeline.cuh"
#include "strategies.cuh"
#include "unionfind.cuh"

namespace rst {

constexpr uint32_t kNoBlock = 0xFFFFFFFFu;
constexpr int kStLevels = 5;  // in-block sparse table: windows of 1..16 positions

// {min of the lo values, max of the hi values} over an index range
struct RmqView {
  const int2* st[kStLevels];  // st[k][i]: indices i .. i+2^k-1 (clipped at the block end)
  const int2* bst;            // level k of the block table at bst + k * nb
  int64_t nb;
};

__device__ __forceinline__ int2 ext(int2 a, int2 b) {
  return make_int2(a.x < b.x ? a.x : b.x, a.y > b.y ? a.y : b.y);
}

// Extremes over indices [l, r] of one 32-index block.
__device__ __forceinline__ int2 rmq_block(const RmqView& v, int64_t l, int64_t r) {
  const int len = (int)(r - l + 1);
  const int k = 31 - __clz(len);
  if (k >= kStLevels)  // the whole block: two windows of 16
    return ext(v.st[kStLevels - 1][l], v.st[kStLevels - 1][l + 16]);
  const int2* t = v.st[0];
#pragma unroll
  for (int j = 1; j < kStLevels; ++j)
    if (k == j) t = v.st[j];  // a select, not a local-memory index
  return ext(t[l], t[r - (1 << k) + 1]);
}

__device__ __forceinline__ int2 rmq(const RmqView& v, int64_t l, int64_t r) {
  const int64_t bl = l >> 5, br = r >> 5;
  if (bl == br) return rmq_block(v, l, r);
  int2 x = ext(rmq_block(v, l, (bl << 5) + 31), rmq_block(v, br << 5, r));
  if (br - bl >= 2) {
    const int64_t b1 = bl + 1, b2 = br - 1;
    const int k = 63 - __clzll(b2 - b1 + 1);
    x = ext(x, ext(v.bst[k * v.nb + b1], v.bst[k * v.nb + b2 - (1LL << k) + 1]));
  }
  return x;
}

// Tour length of every tree: its last arc (the one whose successor was cut)
// has rank len - 1.
__global__ void k_bcc_len(int64_t T, const uint4* __restrict__ pairs, const int32_t* __restrict__ succ,
                          const uint32_t* __restrict__ R, int32_t* __restrict__ lenv) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = pairs[t];  // {i, k, a, b}: i = a->b, k = b->a
    if (succ[r.x] < 0) lenv[r.w] = (int32_t)(R[r.x] + 1);
    if (succ[r.y] < 0) lenv[r.z] = (int32_t)(R[r.y] + 1);
  }
}

__global__ void k_bcc_gather_len(int64_t nroots, const int32_t* __restrict__ roots,
                                 const int32_t* __restrict__ lenv, unsigned long long* __restrict__ tmp) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nroots;
       j += (int64_t)gridDim.x * blockDim.x)
    tmp[j] = (unsigned long long)lenv[roots[j]];
}

// Keys of tree roots; every vertex starts as its own union-find set.
__global__ void k_bcc_root_keys(int64_t nroots, const int32_t* __restrict__ roots,
                                const unsigned long long* __restrict__ base, const int32_t* __restrict__ lenv,
                                int32_t* __restrict__ basev, int32_t* __restrict__ key, int32_t* __restrict__ end) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nroots;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = roots[j];
    const int32_t b = (int32_t)base[j];
    basev[r] = b;
    key[r] = b - 1;
    end[r] = b + lenv[r] - 1;
  }
}

// Keys of non-root vertices from the ranks of their two tree arcs.
__global__ void k_bcc_keys(int64_t T, const uint4* __restrict__ pairs, const uint32_t* __restrict__ R,
                           const int32_t* __restrict__ lab, const int32_t* __restrict__ basev,
                           int32_t* __restrict__ key, int32_t* __restrict__ end) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = pairs[t];
    const int32_t b = basev[lab[r.z]];
    const int32_t gi = b + (int32_t)R[r.x], gk = b + (int32_t)R[r.y];
    if (gi < gk) {  // a->b descends: b is the child
      key[r.w] = gi;
      end[r.w] = gk;
    } else {
      key[r.z] = gk;
      end[r.z] = gi;
    }
  }
}

__global__ void k_bcc_init(int64_t n, const int32_t* __restrict__ key, int32_t* __restrict__ lo,
                           int32_t* __restrict__ hi, int32_t* __restrict__ uf, uint32_t* __restrict__ bmin,
                           uint8_t* __restrict__ cut) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    lo[v] = key[v];
    hi[v] = key[v];
    uf[v] = (int32_t)v;
    bmin[v] = kNoBlock;
    if (cut) cut[v] = 0;
  }
}

// Non-tree arcs: local low/high of the source (one atomic per run of equal
// sources in a warp) and the unrelated-endpoints rule of the auxiliary graph.
template <class OffT>
__global__ void __launch_bounds__(kArcThreads) k_bcc_local(const OffT* __restrict__ off,
                                                           const int32_t* __restrict__ col, int64_t n,
                                                           int64_t A, const int32_t* __restrict__ tile_row,
                                                           const uint32_t* __restrict__ bits,
                                                           const int32_t* __restrict__ key,
                                                           const int32_t* __restrict__ end,
                                                           int32_t* __restrict__ lo, int32_t* __restrict__ hi,
                                                           int32_t* uf, uint32_t* status) {
  __shared__ __align__(16) int32_t s_row[kArcTile];
  const int lane = threadIdx.x & 31;
  for (int64_t a0 = (int64_t)blockIdx.x * kArcTile; a0 < A; a0 += (int64_t)gridDim.x * kArcTile) {
    const int cnt = (int)(A - a0 < kArcTile ? A - a0 : kArcTile);
    const int64_t t = a0 / kArcTile;
    arc_tile_rows(off, n, a0, cnt, s_row, tile_row[t], tile_row[t + 1]);
#pragma unroll 1
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      int32_t x = -1, ky = 0;
      if (i < cnt) {
        const int64_t a = a0 + i;
        const int32_t y = col[a];
        const int32_t u = s_row[i];
        const bool tree = (bits[a >> 5] >> (a & 31)) & 1u;
        if (!tree && y != u && y >= 0 && (int64_t)y < n) {
          x = u;
          ky = key[y];
          if (u < y) {
            const int32_t ku = key[u], eu = end[u], ey = end[y];
            const bool related = (ku <= ky && ky <= eu) || (ky <= ku && ku <= ey);
            if (!related) uf_link(uf, u, y, n, status);
          }
        }
      }
      // segmented min/max over runs of equal sources (the lanes hold
      // consecutive arcs, so equal sources are contiguous): after the
      // doubling steps the first lane of a run holds the run's extremes
      int32_t mn = ky, mx = ky;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t xo = __shfl_down_sync(0xffffffffu, x, d);
        const int32_t mno = __shfl_down_sync(0xffffffffu, mn, d);
        const int32_t mxo = __shfl_down_sync(0xffffffffu, mx, d);
        if (lane + d < 32 && xo == x) {
          mn = mno < mn ? mno : mn;
          mx = mxo > mx ? mxo : mx;
        }
      }
      const int32_t xprev = __shfl_up_sync(0xffffffffu, x, 1);
      if (x >= 0 && (lane == 0 || xprev != x)) {
        if (mn < __ldcg(&lo[x])) atomicMin(&lo[x], mn);
        if (mx > __ldcg(&hi[x])) atomicMax(&hi[x], mx);
      }
    }
    __syncthreads();
  }
}

__global__ void k_fill_i32_pair(int64_t P, int32_t* __restrict__ a, int32_t va, int32_t* __restrict__ b,
                                int32_t vb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = va;
    b[i] = vb;
  }
}

// Bitmap of down-arc positions (the keys of non-root vertices).
__global__ void k_bcc_mark(int64_t n, const int32_t* __restrict__ parent, const int32_t* __restrict__ key,
                           uint32_t* __restrict__ dbits) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (parent[v] == (int32_t)v) continue;  // roots and isolated vertices
    const uint32_t k = (uint32_t)key[v];
    atomicOr(&dbits[k >> 5], 1u << (k & 31));
  }
}

// Preorder index of every non-root vertex and its {lo, hi} at that index.
__global__ void k_bcc_place(int64_t n, const int32_t* __restrict__ parent, const int32_t* __restrict__ key,
                            const uint32_t* __restrict__ dbits, const uint32_t* __restrict__ dpre,
                            const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                            int32_t* __restrict__ idx, int2* __restrict__ m) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (parent[v] == (int32_t)v) continue;
    const uint32_t i = bit_rank(dbits, dpre, (uint64_t)key[v]);
    idx[v] = (int32_t)i;
    m[i] = make_int2(lo[v], hi[v]);
  }
}

struct StPtrs {
  int2* st[kStLevels];
};

// In-block sparse tables (levels 1..4) and the block extremes, one warp per
// 32-index block.
__global__ void k_bcc_st(int64_t P, StPtrs sp, int2* __restrict__ bm) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < P; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int2 a = i < P ? sp.st[0][i] : make_int2(INT_MAX, INT_MIN);
#pragma unroll
    for (int k = 1; k <= kStLevels; ++k) {
      const int d = 1 << (k - 1);
      const int2 o = make_int2(__shfl_down_sync(0xffffffffu, a.x, d), __shfl_down_sync(0xffffffffu, a.y, d));
      if (lane + d < 32) a = ext(a, o);
      if (k < kStLevels && i < P) sp.st[k][i] = a;
    }
    if (lane == 0 && i < P) bm[i >> 5] = a;
  }
}

// Level k of the block table from level k-1 (windows of 2^k blocks, clipped).
__global__ void k_bcc_bst(int64_t nb, int k, int2* __restrict__ b) {
  const int64_t h = 1LL << (k - 1);
  const int2* prev = b + (int64_t)(k - 1) * nb;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j2 = j + h < nb ? j + h : nb - 1;
    b[(int64_t)k * nb + j] = ext(prev[j], prev[j2]);
  }
}

__global__ void k_fill_int2(int64_t P, int2* __restrict__ a, int2 v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// Tree edge u-w (u = parent of w, u not a root) joins w and u when w's
// subtree reaches outside u's subtree.
__global__ void k_bcc_rule2(int64_t n, const int32_t* __restrict__ parent, const int32_t* __restrict__ key,
                            const int32_t* __restrict__ end, const int32_t* __restrict__ idx,
                            const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, RmqView v,
                            int32_t* uf, uint32_t* status) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = parent[w];
    if (u == (int32_t)w || parent[u] == u) continue;
    const int32_t kw = key[w], ew = end[w];
    int2 lh;
    if (ew == kw + 1) {
      lh = make_int2(lo[w], hi[w]);  // a leaf: its subtree is itself
    } else {
      const int64_t l = idx[w], nd = ((int64_t)ew - kw + 1) / 2;
      lh = rmq(v, l, l + nd - 1);
    }
    if (lh.x < key[u] || lh.y > end[u]) uf_link(uf, (int32_t)w, u, n, status);
  }
}

// Block of every arc (its representative vertex, in `label` for now) and the
// smallest arc position per block.  Most tiles lie in one block: the tile
// reduces the positions of the block of its first arc and offers one value;
// arcs of other blocks offer their own.
template <class OffT>
__global__ void __launch_bounds__(kArcThreads) k_bcc_arcblk(const OffT* __restrict__ off,
                                                            const int32_t* __restrict__ col, int64_t n,
                                                            int64_t A, const int32_t* __restrict__ tile_row,
                                                            const uint32_t* __restrict__ bits,
                                                            const int32_t* __restrict__ parent,
                                                            const int32_t* __restrict__ key,
                                                            const int32_t* __restrict__ uf,
                                                            uint32_t* __restrict__ label,
                                                            uint32_t* __restrict__ bmin) {
  __shared__ __align__(16) int32_t s_row[kArcTile];
  __shared__ int32_t s_b0;
  __shared__ uint32_t s_min[kArcThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t a0 = (int64_t)blockIdx.x * kArcTile; a0 < A; a0 += (int64_t)gridDim.x * kArcTile) {
    const int cnt = (int)(A - a0 < kArcTile ? A - a0 : kArcTile);
    const int64_t t = a0 / kArcTile;
    arc_tile_rows(off, n, a0, cnt, s_row, tile_row[t], tile_row[t + 1]);
    int32_t blk[kArcPer];
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      blk[k] = -1;
      if (i < cnt) {
        const int64_t a = a0 + i;
        const int32_t y = col[a], x = s_row[i];
        if (y != x && y >= 0 && (int64_t)y < n) {
          int32_t c;
          if ((bits[a >> 5] >> (a & 31)) & 1u)
            c = parent[y] == x ? y : x;  // tree arc: the child names the edge
          else
            c = key[x] > key[y] ? x : y;  // non-tree: the endpoint met later
          blk[k] = uf[c];
        }
        label[a] = blk[k] >= 0 ? (uint32_t)blk[k] : kNoBlock;
      }
    }
    if (threadIdx.x == 0) s_b0 = blk[0];
    __syncthreads();
    const int32_t b0 = s_b0;
    uint32_t m0 = kNoBlock;
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      if (blk[k] < 0) continue;
      const uint32_t pos = (uint32_t)(a0 + k * kArcThreads + threadIdx.x);
      if (blk[k] == b0) {
        m0 = pos < m0 ? pos : m0;
      } else if (pos < __ldcg(&bmin[blk[k]])) {
        atomicMin(&bmin[blk[k]], pos);
      }
    }
    for (int d = 16; d > 0; d >>= 1) {
      const uint32_t o = __shfl_down_sync(0xffffffffu, m0, d);
      m0 = o < m0 ? o : m0;
    }
    if (lane == 0) s_min[warp] = m0;
    __syncthreads();
    if (threadIdx.x == 0 && b0 >= 0) {
      uint32_t m = kNoBlock;
      for (int w = 0; w < kArcThreads / 32; ++w) m = s_min[w] < m ? s_min[w] : m;
      if (m < __ldcg(&bmin[b0])) atomicMin(&bmin[b0], m);
    }
    __syncthreads();
  }
}

__global__ void k_bcc_label(int64_t A, uint32_t* __restrict__ label, const uint32_t* __restrict__ bmin) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A;
       a += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = label[a];
    if (b != kNoBlock) label[a] = bmin[b];
  }
}

// A vertex is a cut vertex iff two of its arcs (self-loops aside) carry
// different labels, i.e. iff some arc's label differs from the previous
// labelled arc of the same row.
template <class OffT>
__global__ void __launch_bounds__(kArcThreads) k_bcc_cut(const OffT* __restrict__ off, int64_t n, int64_t A,
                                                         const int32_t* __restrict__ tile_row,
                                                         const uint32_t* __restrict__ label,
                                                         uint8_t* __restrict__ cut) {
  __shared__ __align__(16) int32_t s_row[kArcTile];
  for (int64_t a0 = (int64_t)blockIdx.x * kArcTile; a0 < A; a0 += (int64_t)gridDim.x * kArcTile) {
    const int cnt = (int)(A - a0 < kArcTile ? A - a0 : kArcTile);
    const int64_t t = a0 / kArcTile;
    arc_tile_rows(off, n, a0, cnt, s_row, tile_row[t], tile_row[t + 1]);
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      if (i >= cnt) continue;
      const int64_t a = a0 + i;
      const uint32_t L = label[a];
      if (L == kNoBlock) continue;
      const int32_t x = s_row[i];
      const int64_t start = (int64_t)off[x];
      int64_t p = a - 1;
      while (p >= start && label[p] == kNoBlock) --p;  // skip self-loops
      if (p >= start && label[p] != L) cut[x] = 1;
    }
    __syncthreads();
  }
}

__global__ void k_bcc_count(int64_t n, const uint32_t* __restrict__ bmin, unsigned long long* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    const bool b = v < n && bmin[v] != kNoBlock;
    block_reserve<kBlock>(cnt, b ? 1u : 0u);
  }
}

template <class OffT>
size_t bcc_workspace_bytes(int64_t n, int64_t A) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  const int64_t T = n, P = 2 * T, nb = (T + 31) / 32 + 1;
  int levels = 1;
  while ((1LL << levels) <= nb) ++levels;
  size_t b = cc_workspace_bytes<OffT>(n, A) + euler_cc_workspace_bytes(n, A, n, n / 2 + 1);
  b += al((size_t)(n + 1) * 4) * 10;                   // parent, R part, labels, lenv, basev, key, end, lo, hi, uf
  b += al((size_t)P * 4);                              // ranks
  b += al((size_t)(n / 2 + 2) * 8) * 2 + al(scan_tmp_words(n / 2 + 2) * 8);
  b += al((size_t)n * 4);                              // bmin
  b += kStLevels * al((size_t)T * 8);                  // in-block tables of {lo, hi}
  b += al((size_t)levels * nb * 8);                    // block table
  b += 2 * al((size_t)(P / 32 + 2) * 4) + al(scan_tmp_words(P / 32 + 1) * 8) + al((size_t)n * 4);
  b += al((size_t)(A / kArcTile + 2) * 4) + al(64);
  return b;
}

template <class OffT>
rst_status bcc_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A, uint32_t* label,
                   uint8_t* cut, int64_t* nblocks, cudaStream_t s) {
  uint32_t* status = state().status;
  int32_t* lab = ar.take<int32_t>(n);
  int32_t* parent = ar.take<int32_t>(n);
  if (!lab || !parent) return RST_ERR_OOM;
  CcOut cc;
  RST_TRY(cc_run<OffT>(ar, off, col, n, A, 0, lab, &cc, s));
  const int64_t T = cc.T;
  uint32_t* R = ar.take<uint32_t>(2 * T > 0 ? 2 * T : 1);
  if (!R) return RST_ERR_OOM;
  const int32_t* succ = nullptr;
  RST_TRY(euler_root_cc<OffT>(ar, off, n, A, 0, &cc, parent, R, s, &succ));
  prof_mark(s, "bcc_forest");
  const int64_t P = 2 * T;
  int32_t* lenv = ar.take<int32_t>(n);
  int32_t* basev = ar.take<int32_t>(n);
  int32_t* key = ar.take<int32_t>(n);
  int32_t* end = ar.take<int32_t>(n);
  int32_t* lo = ar.take<int32_t>(n);
  int32_t* hi = ar.take<int32_t>(n);
  int32_t* uf = ar.take<int32_t>(n);
  uint32_t* bmin = ar.take<uint32_t>(n);
  const int64_t nr = cc.nroots;
  unsigned long long* base = ar.take<unsigned long long>(nr + 1);
  unsigned long long* stmp = ar.take<unsigned long long>(scan_tmp_words(nr + 1));
  const int64_t tiles = (A + kArcTile - 1) / kArcTile;
  int32_t* tile_row = ar.take<int32_t>(tiles + 2);
  unsigned long long* cnt = ar.take<unsigned long long>(8);
  if (!lenv || !basev || !key || !end || !lo || !hi || !uf || !bmin || !base || !stmp || !tile_row || !cnt)
    return RST_ERR_OOM;
  const int gN = grid_for(n);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  RST_LAUNCH(k_fill_i32_pair, gN, kBlock, 0, s)(n, key, -1, end, -2);  // isolated vertices: never used
  if (T > 0) {
    RST_LAUNCH(k_bcc_len, grid_for(T), kBlock, 0, s)(T, cc.pairs, succ, R, lenv);
    RST_LAUNCH(k_bcc_gather_len, grid_for(nr), kBlock, 0, s)(nr, cc.roots, lenv, base);
    RST_TRY(scan_exclusive_u64(base, base, nr, stmp, s));
    RST_LAUNCH(k_bcc_root_keys, grid_for(nr), kBlock, 0, s)(nr, cc.roots, base, lenv, basev, key, end);
    RST_LAUNCH(k_bcc_keys, grid_for(T), kBlock, 0, s)(T, cc.pairs, R, lab, basev, key, end);
  }
  RST_LAUNCH(k_bcc_init, gN, kBlock, 0, s)(n, key, lo, hi, uf, bmin, cut);
  prof_mark(s, "bcc_keys");
  if (A > 0) {
    RST_LAUNCH(k_arc_tile_rows<OffT>, grid_for(tiles + 1), kBlock, 0, s)(off, n, A, tiles, tile_row);
    if (T > 0)
      RST_LAUNCH(k_bcc_local<OffT>, (unsigned)tiles, kArcThreads, 0, s)(off, col, n, A, tile_row, cc.bits, key,
                                                                       end, lo, hi, uf, status);
  }
  prof_mark(s, "k_bcc_local");
  if (T > 0) {
    // preorder indices of the T non-root vertices and range tables over them
    const int64_t W = P / 32 + 1;
    uint32_t* dbits = ar.take<uint32_t>(W + 1);
    uint32_t* dpre = ar.take<uint32_t>(W + 1);
    unsigned long long* wtmp = ar.take<unsigned long long>(scan_tmp_words(W));
    int32_t* idx = ar.take<int32_t>(n);
    const int64_t nb = (T + 31) / 32;
    int levels = 1;
    while ((1LL << levels) <= nb) ++levels;
    StPtrs sp;
    for (int k = 0; k < kStLevels; ++k) {
      sp.st[k] = ar.take<int2>(T);
      if (!sp.st[k]) return RST_ERR_OOM;
    }
    int2* bst = ar.take<int2>((int64_t)levels * nb);
    if (!dbits || !dpre || !wtmp || !idx || !bst) return RST_ERR_OOM;
    RST_CUDA(cudaMemsetAsync(dbits, 0, (W + 1) * sizeof(uint32_t), s));
    RST_LAUNCH(k_bcc_mark, gN, kBlock, 0, s)(n, parent, key, dbits);
    RST_TRY(scan_popcount_words(dbits, dpre, W, wtmp, s));
    RST_LAUNCH(k_fill_int2, grid_for(T), kBlock, 0, s)(T, sp.st[0], make_int2(INT_MAX, INT_MIN));
    RST_LAUNCH(k_bcc_place, gN, kBlock, 0, s)(n, parent, key, dbits, dpre, lo, hi, idx, sp.st[0]);
    RST_LAUNCH(k_bcc_st, grid_for(T), kBlock, 0, s)(T, sp, bst);
    for (int k = 1; k < levels; ++k) RST_LAUNCH(k_bcc_bst, grid_for(nb), kBlock, 0, s)(nb, k, bst);
    prof_mark(s, "bcc_tables");
    RmqView v;
    for (int k = 0; k < kStLevels; ++k) v.st[k] = sp.st[k];
    v.bst = bst;
    v.nb = nb;
    RST_LAUNCH(k_bcc_rule2, gN, kBlock, 0, s)(n, parent, key, end, idx, lo, hi, v, uf, status);
    prof_mark(s, "k_bcc_rule2");
  }
  RST_LAUNCH(k_uf_compress, gN, kBlock, 0, s)(n, uf, status);
  if (A > 0) {
    RST_LAUNCH(k_bcc_arcblk<OffT>, (unsigned)tiles, kArcThreads, 0, s)(off, col, n, A, tile_row, cc.bits, parent,
                                                                      key, uf, label, bmin);
    RST_LAUNCH(k_bcc_label, grid_for(A), kBlock, 0, s)(A, label, bmin);
    if (cut) RST_LAUNCH(k_bcc_cut<OffT>, (unsigned)tiles, kArcThreads, 0, s)(off, n, A, tile_row, label, cut);
  }
  RST_LAUNCH(k_bcc_count, gN, kBlock, 0, s)(n, bmin, cnt);
  prof_mark(s, "bcc_labels");
  RST_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  RST_TRY(fetch_u64(cnt, 1, &h, s));
  if (nblocks) *nblocks = (int64_t)h;
  return RST_OK;
}

template size_t bcc_workspace_bytes<int32_t>(int64_t, int64_t);
template size_t bcc_workspace_bytes<int64_t>(int64_t, int64_t);
template rst_status bcc_run<int32_t>(Arena&, const int32_t*, const int32_t*, int64_t, int64_t, uint32_t*,
                                     uint8_t*, int64_t*, cudaStream_t);
template rst_status bcc_run<int64_t>(Arena&, const int64_t*, const int32_t*, int64_t, int64_t, uint32_t*,
                                     uint8_t*, int64_t*, cudaStream_t);

}  // namespace rst
