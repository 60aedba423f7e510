// Euler-tour rooting of a spanning forest (Section III-D).
//
// Tree arcs are addressed by their place in lexicographic (src, dst) order
// ("tree positions").  With the CSR-bitmap front end that order needs no sort:
// the CSR rows are already sorted, so the tree arcs in CSR order ARE the
// lexicographically sorted arc array, and the tree position of CSR position j
// is the number of marked bits before j (a popcount prefix over the bitmap).
// A vertex's tree arcs form one run of consecutive tree positions, and
// next(e) = e+1 inside a run.
//
// succ(e) = next(rev(e)) if rev(e) is not the last arc of its run, otherwise
// first(from(rev(e))).  For every tree root r the arc e with rev(e) = last[r]
// gets succ(e) = -1, turning each tree's Euler cycle into a list with head
// first[r].  After list ranking, of the twins e = a->b and rev(e) = b->a the
// one ranked first descends from parent to child.
#include "pipeline.cuh"

namespace rst {

// ----------------------------------------------------------------- core

// Tree records per thread and step in leaf pruning, whose byte gathers are
// issued together so several dependent chains are in flight (the other record
// kernels are bound by DRAM sectors and gain nothing from it).
constexpr int kEuPer = 4;
constexpr int kEuBlocksPerSm = 6;  // resident blocks at its 40 registers

__global__ void k_parent_from_rank(int64_t T, const uint4* __restrict__ pairs,
                                   const uint32_t* __restrict__ R, int32_t* __restrict__ parent) {
  pdl_wait();  // launched as a programmatic dependent
  const uint64_t once = l2_evict_first();  // the records: read once, keep L2 for R and parent
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = ld_stream(&pairs[t], once);  // {i, k, a, b}: i = a->b, k = b->a
    if (r.x == kNone) continue;  // a pruned leaf edge: parent already set
    const uint32_t ri = R[r.x], rk = R[r.y];
    if (ri < rk)
      parent[r.w] = (int32_t)r.z;  // a->b traversed first: a is b's parent
    else
      parent[r.z] = (int32_t)r.w;
  }
}

// The same with positions read from the first list-ranking level's records
// (the final pass over all elements left out); it also reports a walk that did
// not reach every element (the input was not a forest).
__global__ void k_parent_from_owner(int64_t T, const uint4* __restrict__ pairs, const int2* __restrict__ ol,
                                    const uint32_t* __restrict__ ol32, int fbits,
                                    const uint32_t* __restrict__ spos, int64_t S,
                                    const unsigned long long* visited, int64_t N,
                                    int32_t* __restrict__ parent, uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  if (visited && blockIdx.x == 0 && threadIdx.x == 0 && *visited != (unsigned long long)N)
    raise_error(status, DERR_NOT_FOREST);
  const uint64_t once = l2_evict_first();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = ld_stream(&pairs[t], once);  // {i, k, a, b}: i = a->b, k = b->a
    if (r.x == kNone) continue;
    const uint32_t ri = lr_position(ol, ol32, fbits, spos, S, r.x);
    const uint32_t rk = lr_position(ol, ol32, fbits, spos, S, r.y);
    if (ri < rk)
      parent[r.w] = (int32_t)r.z;
    else
      parent[r.z] = (int32_t)r.w;
  }
}

static size_t euler_core_bytes(int64_t T) {
  const int64_t N = 2 * T;
  return ((size_t)N * 8 + 255) / 256 * 256 + 256 + ((size_t)N * 4 + 255) / 256 * 256 + 256 +
         list_rank_workspace_upper(N);
}

// ----------------------------------------------------------------- CSR-bitmap front end

// Tree root of the component with canonical label L: the requested root of
// that component, else L (its minimum vertex).
__device__ __forceinline__ int32_t tree_root_for(int32_t L, int32_t root_label, int32_t root,
                                                 const int32_t* __restrict__ rootof) {
  if (rootof) {
    const int32_t r = rootof[L];
    return r >= 0 ? r : L;
  }
  return L == root_label ? root : L;
}

__global__ void k_mark_roots(int64_t nroots, const int32_t* __restrict__ roots, int32_t root_label,
                             int32_t root, const int32_t* __restrict__ rootof,
                             uint32_t* __restrict__ root_bits) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nroots;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = tree_root_for(roots[k], root_label, root, rootof);
    atomicOr(&root_bits[r >> 5], 1u << (r & 31));
  }
}

__device__ __forceinline__ bool is_tree_root(const uint32_t* __restrict__ root_bits, int64_t v) {
  return (root_bits[v >> 5] >> (v & 31)) & 1u;
}

// ----------------------------------------------------------------- row starts

int64_t row_start_words(int64_t A) { return A / 32 + 2; }

template <class OffT>
__global__ void k_row_starts(const OffT* __restrict__ off, int64_t n, uint32_t* __restrict__ rs) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base <= n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    row_start_bit(rs, off, n, v, v <= n ? (uint64_t)off[v] : 0, v < n ? (uint64_t)off[v + 1] : 0);
  }
}

template <class OffT>
rst_status row_starts(const OffT* off, int64_t n, int64_t A, uint32_t* rs, cudaStream_t s) {
  RST_CUDA(cudaMemsetAsync(rs, 0, row_start_words(A) * sizeof(uint32_t), s));
  RST_LAUNCH(k_row_starts<OffT>, grid_for(n + 1), kBlock, 0, s)(off, n, rs);
  return RST_OK;
}
template rst_status row_starts<int32_t>(const int32_t*, int64_t, int64_t, uint32_t*, cudaStream_t);
template rst_status row_starts<int64_t>(const int64_t*, int64_t, int64_t, uint32_t*, cudaStream_t);

// Words a row-start or tree-bit scan reads before it falls back to the
// vertex's offsets (rows of a few arcs end within one or two words).
constexpr int kRunScanWords = 4;

// For the tree arc at CSR position pos: true iff no tree arc follows it in
// its row, i.e. the next tree bit comes at or after the next row start (a
// position that is both is the next row's first arc).  *ok = false when the
// scan gave up.  Bit A of rs is set, so the scan never passes word A/32.
__device__ __forceinline__ bool last_in_run(const uint2* __restrict__ rk, const uint32_t* __restrict__ rs,
                                            uint64_t pos, bool* ok) {
  uint64_t w = (pos + 1) >> 5;
  uint32_t m = ~0u << ((pos + 1) & 31);
  for (int it = 0; it < kRunScanWords; ++it, ++w, m = ~0u) {
    const uint32_t t = rk[w].x & m, r = rs[w] & m;
    if (t | r) {
      *ok = true;
      if (!r) return false;
      if (!t) return true;
      return __ffs(r) <= __ffs(t);
    }
  }
  *ok = false;
  return false;
}

// Start of the row holding CSR position pos (the last row start at or
// before it); *ok = false when the scan gave up.
__device__ __forceinline__ uint64_t row_start_of(const uint32_t* __restrict__ rs, uint64_t pos, bool* ok) {
  int64_t w = (int64_t)(pos >> 5);
  uint32_t m = (2u << (pos & 31)) - 1u;  // bits 0..pos&31 (all ones for bit 31)
  for (int it = 0; it < kRunScanWords && w >= 0; ++it, --w, m = ~0u) {
    const uint32_t r = rs[w] & m;
    if (r) {
      *ok = true;
      return ((uint64_t)w << 5) + 31u - (uint32_t)__clz(r);
    }
  }
  *ok = false;
  return 0;
}

// Euler successor of the arc that follows the tree arc at CSR position pos
// (tree position tp) in the tour: the next tree arc of v's row, else the
// first one of the row (the wrap), else -1 when v is a tree root (the cut).
template <class OffT>
__device__ __forceinline__ int32_t run_successor(const uint2* __restrict__ rk, const uint32_t* __restrict__ rs,
                                                 const uint32_t* __restrict__ root_bits,
                                                 const OffT* __restrict__ off, uint64_t pos, int32_t v,
                                                 uint32_t tp) {
  bool ok;
  bool last = last_in_run(rk, rs, pos, &ok);
  if (!ok) last = tp + 1u == bit_rank2(rk, (uint64_t)off[v + 1]);
  if (!last) return (int32_t)(tp + 1u);
  if (is_tree_root(root_bits, v)) return -1;
  const uint64_t st = row_start_of(rs, pos, &ok);
  return (int32_t)bit_rank2(rk, ok ? st : (uint64_t)off[v]);
}

// Per vertex, from its tree-arc run [rank(off[v]), rank(off[v+1])): with
// parent set, roots and singletons take P[v] = v; with leaf set, the leaf
// bitmap (n/32 + 1 words) marks vertices of tree degree 1 that are not tree
// roots, one word per warp (a ballot: the warp's 32 vertices are one word).
template <class OffT>
__global__ void k_run_flags(const OffT* __restrict__ off, int64_t n, const uint2* __restrict__ rk,
                            const uint32_t* __restrict__ root_bits, int32_t* __restrict__ parent,
                            uint32_t* __restrict__ leaf) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    bool lf = false;
    if (v < n) {
      const uint32_t t0 = bit_rank2(rk, (uint64_t)off[v]);
      const uint32_t t1 = bit_rank2(rk, (uint64_t)off[v + 1]);
      const bool rt = is_tree_root(root_bits, v);
      if (parent && (t0 == t1 || rt)) parent[v] = (int32_t)v;
      lf = t1 - t0 == 1u && !rt;
    }
    if (leaf) {
      const uint32_t w = __ballot_sync(0xffffffffu, lf);
      if ((threadIdx.x & 31) == 0 && v < n) leaf[v >> 5] = w;
    }
  }
}

__device__ __forceinline__ bool is_leaf(const uint32_t* __restrict__ leaf, uint32_t v) {
  return (__ldg(&leaf[v >> 5]) >> (v & 31)) & 1u;
}

// Leaf pruning (rake) before the tour: a non-root vertex of tree degree 1
// has its single tree neighbour as parent.  Its edge leaves the tree that is
// toured (both arcs' bits are cleared) and the pair is marked done.  Removing
// leaves changes no ancestor relation among the remaining vertices.
__global__ void __launch_bounds__(kBlock, kEuBlocksPerSm) k_prune_leaves(int64_t T, uint4* __restrict__ pairs, const uint32_t* __restrict__ leaf,
                               uint32_t* __restrict__ bits, int32_t* __restrict__ parent) {
  pdl_wait();  // launched as a programmatic dependent
  const int64_t tile = (int64_t)blockDim.x * kEuPer;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < T; base += (int64_t)gridDim.x * tile) {
    uint4 r[kEuPer];
#pragma unroll
    for (int j = 0; j < kEuPer; ++j) {
      const int64_t t = base + (int64_t)j * blockDim.x + threadIdx.x;
      r[j] = t < T ? pairs[t] : make_uint4(0, 0, 0, 0);
    }
    bool la[kEuPer], lb[kEuPer];
#pragma unroll
    for (int j = 0; j < kEuPer; ++j) {
      const int64_t t = base + (int64_t)j * blockDim.x + threadIdx.x;
      la[j] = t < T && is_leaf(leaf, r[j].z);
      lb[j] = t < T && is_leaf(leaf, r[j].w);
    }
#pragma unroll
    for (int j = 0; j < kEuPer; ++j) {
      if (!la[j] && !lb[j]) continue;
      const int64_t t = base + (int64_t)j * blockDim.x + threadIdx.x;
      const int32_t a = (int32_t)r[j].z, b = (int32_t)r[j].w;
      if (lb[j]) parent[b] = a;
      if (la[j]) parent[a] = b;
      atomicAnd(&bits[r[j].x >> 5], ~(1u << (r[j].x & 31)));
      atomicAnd(&bits[r[j].y >> 5], ~(1u << (r[j].y & 31)));
      pairs[t].x = kNone;  // the record's first word marks it done
    }
  }
}

template <class OffT>
__global__ void k_heads(int64_t nroots, const int32_t* __restrict__ roots, int32_t root_label,
                        int32_t root, const int32_t* __restrict__ rootof, const OffT* __restrict__ off,
                        const uint2* __restrict__ rk, int32_t* __restrict__ heads) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nroots;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = tree_root_for(roots[k], root_label, root, rootof);
    const uint32_t t0 = bit_rank2(rk, (uint64_t)off[r]), t1 = bit_rank2(rk, (uint64_t)off[r + 1]);
    heads[k] = t1 > t0 ? (int32_t)t0 : -1;  // -1: nothing left to tour
  }
}

// {p, q, a, b} (CSR positions) -> {i, k, a, b} (tree positions), in place,
// and the Euler successors of both arcs: succ(i) follows rev(i) = k in b's
// run (wrapping to first[b]), succ(k) follows i in a's run; the arc that
// wraps into a tree root's first arc is cut (succ = -1).  Whether an arc is
// the last of its run and where its row starts come from the tree-arc and
// row-start bitmaps (L2-resident), not from the endpoints' offsets.
template <class OffT>
__global__ void k_pairs_succ(int64_t T, uint4* __restrict__ pairs, const uint2* __restrict__ rk,
                             const uint32_t* __restrict__ rs, const uint32_t* __restrict__ root_bits,
                             const OffT* __restrict__ off, int32_t* __restrict__ succ) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint4 r = pairs[t];
    if (r.x == kNone) continue;  // pruned leaf edge
    const uint32_t p = r.x, q = r.y;
    const uint32_t i = bit_rank2(rk, p);
    const uint32_t k = bit_rank2(rk, q);
    const int32_t a = (int32_t)r.z, b = (int32_t)r.w;
    r.x = i;
    r.y = k;
    pairs[t] = r;
    succ[i] = run_successor(rk, rs, root_bits, off, q, b, k);
    succ[k] = run_successor(rk, rs, root_bits, off, p, a, i);
  }
}

size_t euler_cc_workspace_bytes(int64_t n, int64_t A, int64_t T, int64_t nroots) {
  const int64_t W = A / 32 + 1;
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  size_t b = al((W + 1) * 8) + al(scan_tmp_words(W) * 8) + al((n / 32 + 1) * 4) +
             al(row_start_words(A) * 4) + al(n) + al(nroots * 4 + 4) + 256;
  return b + euler_core_bytes(T);
}

template <class OffT>
rst_status euler_root_cc(Arena& ar, const OffT* off, int64_t n, int64_t A, int32_t root, CcOut* cc,
                         int32_t* parent_out, uint32_t* rank_out, cudaStream_t s, const int32_t** succ_view) {
  const int64_t W = A / 32 + 1;
  // the ranked bitmap and the cleared root flags may already be queued by the
  // connectivity pass (cc->rk, cc->root_bits, cc->rs)
  const bool pre = cc->rk != nullptr && cc->rk_tmp != nullptr && cc->root_bits != nullptr && cc->rs != nullptr;
  uint2* rk = pre ? cc->rk : ar.take<uint2>(W + 1);  // {tree-arc bitmap word, prefix}
  unsigned long long* tmp = pre ? cc->rk_tmp : ar.take<unsigned long long>(scan_tmp_words(W));
  uint32_t* root_bits = pre ? cc->root_bits : ar.take<uint32_t>(n / 32 + 1);
  uint32_t* rs = pre ? cc->rs : ar.take<uint32_t>(row_start_words(A));
  int32_t* heads = ar.take<int32_t>(cc->nroots + 1);
  if (!rk || !tmp || !root_bits || !rs || !heads) return RST_ERR_OOM;
  if (!pre) {
    RST_TRY(scan_popcount_ranked(cc->bits, rk, W, tmp, s));
    prof_mark(s, "eu_bitscan");
    RST_CUDA(cudaMemsetAsync(root_bits, 0, (n / 32 + 1) * sizeof(uint32_t), s));
    RST_TRY(row_starts<OffT>(off, n, A, rs, s));
  }
  if (cc->nroots > 0)
    RST_LAUNCH_PDL(k_mark_roots, grid_for(cc->nroots), kBlock, 0, s)(cc->nroots, cc->roots, cc->root_label,
                                                         root, cc->rootof, root_bits);
  prof_mark(s, "eu_roots");
  const int64_t T = cc->T;
  // Without requested ranks the tour only has to order each edge's twins, so
  // leaves are pruned first: their parent is their single tree neighbour.
  const bool prune = rank_out == nullptr && T > 0;
  uint32_t* leaf = prune ? ar.take<uint32_t>(n / 32 + 1) : nullptr;
  if (prune && !leaf) return RST_ERR_OOM;
  // the plain grid-stride kernels of the tour take the tuned block size
  const int eb = tuning().euler_block;
  RST_LAUNCH_PDL((k_run_flags<OffT>), grid_for(n, eb, 2048 / eb), eb, 0, s)(off, n, rk, root_bits, parent_out, leaf);
  prof_mark(s, "k_run_flags");
  int64_t N = 2 * T;
  if (prune) {
    RST_LAUNCH_PDL(k_prune_leaves, grid_for((T + kEuPer - 1) / kEuPer, kBlock, kEuBlocksPerSm), kBlock, 0, s)(T, cc->pairs, leaf, cc->bits, parent_out);
    prof_mark(s, "k_prune_leaves");
    RST_TRY(scan_popcount_ranked(cc->bits, rk, W, tmp, s));
    prof_mark(s, "eu_reduced");
  }
  if (cc->nroots > 0)
    RST_LAUNCH_PDL((k_heads<OffT>), grid_for(cc->nroots), kBlock, 0, s)(cc->nroots, cc->roots, cc->root_label, root,
                                                          cc->rootof, off, rk, heads);
  RST_CUDA(cudaGetLastError());
  if (T <= 0) return RST_OK;
  // The successors need only T (the array holds at most 2T arcs), so they are
  // queued behind the read-back of the pruned arc count: the GPU builds them
  // while the host waits for the count that sizes the ranking levels.
  int32_t* succ = ar.take<int32_t>(N);
  if (!succ) return RST_ERR_OOM;
  cudaEvent_t ev = state().readback;  // none in the fixed-scratch variant: it synchronises the stream
  // pinned read-back word (a copy into pageable memory would block the host)
  unsigned long long* hw = state().hostbuf + 2;
  if (prune) RST_CUDA(cudaMemcpyAsync(hw, &rk[W].y, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (prune && ev) RST_CUDA(cudaEventRecord(ev, s));
  const int gT = grid_for(T, eb, 2048 / eb);
  RST_LAUNCH_PDL((k_pairs_succ<OffT>), gT, eb, 0, s)(T, cc->pairs, rk, rs, root_bits, off, succ);
  prof_mark(s, "k_pairs_succ");
  RST_CUDA(cudaGetLastError());
  if (prune) {
    if (ev)
      RST_CUDA(cudaEventSynchronize(ev));
    else
      RST_CUDA(cudaStreamSynchronize(s));
    uint32_t left32 = 0;
    std::memcpy(&left32, hw, sizeof(uint32_t));
    N = (int64_t)left32;
  }
  if (N <= 0) return RST_OK;
  uint32_t* R = rank_out ? rank_out : ar.take<uint32_t>(N);
  if (!R) return RST_ERR_OOM;
  if (succ_view) *succ_view = succ;  // stays valid while the arena is not reset
  // Without requested ranks the parents read their positions straight from the
  // first ranking level's records (no pass writing every position).
  LrFirstLevel lv;
  RST_TRY(list_rank(ar, N, succ, nullptr, heads, cc->nroots, R, s, rank_out ? nullptr : &lv));
  if (lv.valid) {
    RST_LAUNCH_PDL(k_parent_from_owner, gT, eb, 0, s)(T, cc->pairs, lv.ol, lv.ol32, lv.fbits, lv.spos, lv.S,
                                                      lv.visited, lv.N, parent_out, state().status);
    prof_mark(s, "k_parent_from_owner");
  } else {
    RST_LAUNCH_PDL(k_parent_from_rank, gT, eb, 0, s)(T, cc->pairs, R, parent_out);
    prof_mark(s, "k_parent_from_rank");
  }
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}

template rst_status euler_root_cc<int32_t>(Arena&, const int32_t*, int64_t, int64_t, int32_t, CcOut*,
                                           int32_t*, uint32_t*, cudaStream_t, const int32_t**);
template rst_status euler_root_cc<int64_t>(Arena&, const int64_t*, int64_t, int64_t, int32_t, CcOut*,
                                           int32_t*, uint32_t*, cudaStream_t, const int32_t**);

// ----------------------------------------------------------------- edge-list front end

static int key_bits_for(int64_t n) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < n) ++b;
  return b;
}

__global__ void k_arc_keys(int64_t T, const int32_t* __restrict__ uv, int64_t n, int nb,
                           uint64_t* __restrict__ keys, uint32_t* status) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = uv[2 * t], v = uv[2 * t + 1];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) {
      raise_error(status, DERR_NOT_FOREST);
      u = 0;
      v = 0;  // keys of a rejected edge; the call reports the error
    }
    keys[t] = ((uint64_t)(uint32_t)u << nb) | (uint32_t)v;
    keys[t + T] = ((uint64_t)(uint32_t)v << nb) | (uint32_t)u;
  }
}

__global__ void k_count_src(int64_t N, const uint64_t* __restrict__ keys, int nb,
                            unsigned long long* __restrict__ deg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&deg[keys[i] >> nb], 1ull);
}

__global__ void k_key_dst(int64_t N, const uint64_t* __restrict__ keys, int nb, int32_t* __restrict__ cols) {
  const uint64_t mask = ((uint64_t)1 << nb) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    cols[i] = (int32_t)(keys[i] & mask);
}

size_t euler_edges_workspace_bytes(int64_t n, int64_t T) {
  const int64_t N = 2 * T;
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  size_t b = al(N * 8) + radix_sort_workspace_bytes(N) + al((n + 1) * 8) + al(scan_tmp_words(n + 1) * 8) +
             al(N * 4);
  b += cc_workspace_bytes<int64_t>(n, N);
  b += euler_cc_workspace_bytes(n, N, T, n / 2 + 1);
  return b;
}

rst_status euler_root_edges(Arena& ar, int64_t n, const int32_t* tree_uv, int64_t T, int32_t root,
                            int32_t* parent_out, uint32_t* rank_out, cudaStream_t s) {
  const int64_t N = 2 * T;
  const int nb = key_bits_for(n);
  uint64_t* keys = ar.take<uint64_t>(N);
  unsigned long long* off = ar.take<unsigned long long>(n + 1);
  unsigned long long* tmp = ar.take<unsigned long long>(scan_tmp_words(n + 1));
  int32_t* cols = ar.take<int32_t>(N);
  if (!keys || !off || !tmp || !cols) return RST_ERR_OOM;
  uint32_t* status = state().status;
  if (T > 0) {
    RST_LAUNCH(k_arc_keys, grid_for(T), kBlock, 0, s)(T, tree_uv, n, nb, keys, status);
    RST_TRY(radix_sort_keys(ar, keys, N, 2 * nb, s));
  }
  RST_CUDA(cudaMemsetAsync(off, 0, (n + 1) * sizeof(unsigned long long), s));
  if (T > 0) {
    RST_LAUNCH(k_count_src, grid_for(N), kBlock, 0, s)(N, keys, nb, off);
    RST_LAUNCH(k_key_dst, grid_for(N), kBlock, 0, s)(N, keys, nb, cols);
  }
  RST_TRY(scan_exclusive_u64(off, off, n, tmp, s));
  RST_CUDA(cudaGetLastError());
  RST_TRY(read_device_error(s));
  const int64_t* off64 = reinterpret_cast<const int64_t*>(off);
  CcOut cc;
  RST_TRY(cc_run<int64_t>(ar, off64, cols, n, N, root, nullptr, &cc, s));
  if (cc.T != T) return RST_ERR_DEVICE;  // a cycle or a repeated edge: not a forest
  return euler_root_cc<int64_t>(ar, off64, n, N, root, &cc, parent_out, rank_out, s);
}

}  // namespace rst
