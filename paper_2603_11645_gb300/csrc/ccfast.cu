// Fast non-deterministic spanning forest: sampled union-find with CAS hooking
// (the hooking freedom Section III-B leaves: any rule that merges components
// works; this one trades the deterministic minimum-key forest for less work).
//
//  1 first neighbours: the atomic-free round 1 of the deterministic path
//    (every vertex hooks to the first entry of its sorted row; mutual pairs
//    are the roots) gives a forest whose roots are its trees' minimum
//    vertices, the tree-edge records with their twin arcs, and P pointing at
//    the roots, which is a ready union-find state;
//  2 sampling: every vertex links with the second entry of its row (link =
//    find both roots, CAS the larger root's pointer to the smaller one); one
//    successful CAS merges two trees, so the arc that made it is a
//    spanning-forest edge and is recorded; then every pointer is compressed;
//  3 the most frequent root among a fixed sample of vertices is the giant
//    component; vertices outside it link with the rest of their rows (an edge
//    from the giant to another component is met from the other side);
//  4 compress again.  Hooking the larger root under the smaller keeps every
//    root the minimum vertex of its set: the roots are the canonical labels.
//  5 every recorded edge {u, v} (arc p = u->v) finds its twin q = v->u by a
//    binary search in v's sorted row; both arcs are marked in the CSR bitmap
//    and the record {p, q, u, v} feeds the Euler-tour rooting unchanged.
//
// Races only decide WHICH edge merges two trees; every run returns a valid
// spanning forest with the same components (and the same tree roots).  All
// union-find reads go to L2 (__ldcg): a stale L1 copy of a root pointer would
// make the CAS fail again and again.  Every loop is bounded.
#include "csr_walk.cuh"
#include "pipeline.cuh"
#include "strategies.cuh"
#include "unionfind.cuh"

namespace rst {

constexpr int kSampleRounds = 2;  // row entries 0 and 1 are linked for every vertex
constexpr int kGiantSample = 1024;

// counters: round-1 records (the index round 1 counts in), roots, the giant
// root, the requested root's label, union-find tree edges
enum { FC_R1 = 0, FC_ROOTS = 1, FC_GIANT_ROOT = 2, FC_ROOT_LABEL = 3, FC_TREE = 4 };

// Round r of the sampling: vertex u links with the r-th entry of its row.
template <class OffT>
__global__ void k_fast_sample(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                              int r, int32_t* uf, int3* __restrict__ tl, unsigned long long* cnt,
                              int64_t cap, uint32_t* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t u = base + threadIdx.x;
    bool rec = false;
    int3 e = make_int3(0, 0, 0);
    if (u < n) {
      const int64_t p = (int64_t)off[u] + r;
      if (p < (int64_t)off[u + 1]) {
        const int32_t v = col[p];
        if (v < 0 || (int64_t)v >= n) {
          raise_error(status, DERR_INDEX);
        } else if (v != (int32_t)u && uf_link(uf, (int32_t)u, v, n, status)) {
          rec = true;
          e = make_int3((int32_t)p, (int32_t)u, v);
        }
      }
    }
    const unsigned long long slot = block_reserve<kBlock>(&cnt[FC_TREE], rec ? 1u : 0u);
    if (rec) {
      if ((int64_t)slot < cap)
        tl[slot] = e;
      else
        raise_error(status, DERR_CAPACITY);
    }
  }
}

__global__ void k_uf_compress(int64_t n, int32_t* uf, uint32_t* status) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    uf[v] = uf_root(uf, (int32_t)v, n, status);
}

// The giant component: the most frequent root among kGiantSample vertices
// spread evenly over the ids (ties: the smaller root).  One block.
__global__ void k_fast_giant(int64_t n, const int32_t* __restrict__ uf, unsigned long long* cnt) {
  __shared__ int32_t s_lab[kGiantSample];
  __shared__ unsigned long long s_best;
  const int k = n < kGiantSample ? (int)n : kGiantSample;
  for (int i = threadIdx.x; i < k; i += blockDim.x) s_lab[i] = __ldcg(&uf[(int64_t)i * n / k]);
  if (threadIdx.x == 0) s_best = ~0ull;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int c = 0;
    for (int j = 0; j < k; ++j) c += s_lab[j] == s_lab[i];
    // larger count first, then smaller root
    const unsigned long long key = ((unsigned long long)(kGiantSample - c) << 32) | (uint32_t)s_lab[i];
    atomicMin(&s_best, key);
  }
  __syncthreads();
  if (threadIdx.x == 0) cnt[FC_GIANT_ROOT] = k > 0 ? (s_best & 0xffffffffull) : ~0ull;
}

// Vertices outside the giant component link with the rest of their rows.
template <class OffT>
__global__ void k_fast_rest(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                            int32_t* uf, int3* __restrict__ tl, unsigned long long* cnt, int64_t cap,
                            uint32_t* status) {
  const int32_t giant = (int32_t)cnt[FC_GIANT_ROOT];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(&uf[u]) == giant) continue;  // compressed: uf[u] is u's root
    const int64_t end = (int64_t)off[u + 1];
    for (int64_t p = (int64_t)off[u] + kSampleRounds; p < end; ++p) {
      const int32_t v = col[p];
      if (v < 0 || (int64_t)v >= n) {
        raise_error(status, DERR_INDEX);
        break;
      }
      if (v != (int32_t)u && uf_link(uf, (int32_t)u, v, n, status)) {
        const unsigned long long slot = atomicAdd(&cnt[FC_TREE], 1ull);
        if ((int64_t)slot < cap)
          tl[slot] = make_int3((int32_t)p, (int32_t)u, v);
        else
          raise_error(status, DERR_CAPACITY);
      }
    }
  }
}

// Tree-edge records (after round 1's) and bitmap marks of the union-find
// edges; roots of components with edges.
template <class OffT>
__global__ void k_fast_pairs(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                             const int3* __restrict__ tl, const unsigned long long* cnt,
                             uint4* __restrict__ pairs0, uint32_t* __restrict__ bits, uint32_t* status) {
  const int64_t T = (int64_t)cnt[FC_TREE];
  uint4* __restrict__ pairs = pairs0 + cnt[FC_R1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int3 e = tl[t];
    const int64_t q = row_find(off, col, e.z, e.y);
    if (q < 0) {
      raise_error(status, DERR_INDEX);  // the CSR is not symmetric
      continue;
    }
    pairs[t] = make_uint4((uint32_t)e.x, (uint32_t)q, (uint32_t)e.y, (uint32_t)e.z);
    atomicOr(&bits[(uint32_t)e.x >> 5], 1u << ((uint32_t)e.x & 31));
    atomicOr(&bits[(uint64_t)q >> 5], 1u << ((uint32_t)q & 31));
  }
}

template <class OffT>
__global__ void k_fast_roots(const OffT* __restrict__ off, int64_t n, const int32_t* __restrict__ uf,
                             int32_t root, int32_t* __restrict__ roots, unsigned long long* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    bool r = false;
    if (v < n) {
      const int32_t L = uf[v];
      r = L == (int32_t)v && off[v + 1] > off[v];
      if (v == root) cnt[FC_ROOT_LABEL] = (unsigned long long)(uint32_t)L;
    }
    const unsigned long long slot = block_reserve<kBlock>(&cnt[FC_ROOTS], r ? 1u : 0u);
    if (r) roots[slot] = (int32_t)v;
  }
}

template <class OffT>
size_t ccfast_workspace_bytes(int64_t n, int64_t A) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  return 2 * al((size_t)n * 4) + al((size_t)n * 12) + al((size_t)n * 16) + al(((size_t)A / 32 + 2) * 4) +
         al((size_t)(n / 2 + 1) * 4) + al(8 * 8);
}

template <class OffT>
rst_status ccfast_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                      int32_t* labels_out, CcOut* out, cudaStream_t s) {
  int32_t* uf = ar.take<int32_t>(n);
  uint32_t* J = ar.take<uint32_t>(n);
  int3* tl = ar.take<int3>(n);
  uint4* pairs = ar.take<uint4>(n);
  uint32_t* bits = ar.take<uint32_t>(A / 32 + 2);
  int32_t* roots = ar.take<int32_t>(n / 2 + 1);
  unsigned long long* cnt = ar.take<unsigned long long>(8);
  if (!uf || !J || !tl || !pairs || !bits || !roots || !cnt) return RST_ERR_OOM;
  uint32_t* status = state().status;
  const int gN = grid_for(n);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  RST_CUDA(cudaMemsetAsync(bits, 0, (A / 32 + 2) * sizeof(uint32_t), s));
  prof_mark(s, "fast_setup");
  RST_TRY(round1_forest<OffT>(off, col, n, uf, J, pairs, bits, cnt, s));
  prof_mark(s, "fast_round1");
  RST_LAUNCH(k_fast_sample<OffT>, gN, kBlock, 0, s)(off, col, n, 1, uf, tl, cnt, n, status);
  prof_mark(s, "k_fast_sample");
  RST_LAUNCH(k_uf_compress, gN, kBlock, 0, s)(n, uf, status);
  RST_LAUNCH(k_fast_giant, 1, kBlock, 0, s)(n, uf, cnt);
  prof_mark(s, "k_fast_compress");
  RST_LAUNCH(k_fast_rest<OffT>, gN, kBlock, 0, s)(off, col, n, uf, tl, cnt, n, status);
  prof_mark(s, "k_fast_rest");
  RST_LAUNCH(k_uf_compress, gN, kBlock, 0, s)(n, uf, status);
  RST_LAUNCH(k_fast_roots<OffT>, gN, kBlock, 0, s)(off, n, uf, root, roots, cnt);
  RST_LAUNCH(k_fast_pairs<OffT>, gN, kBlock, 0, s)(off, col, tl, cnt, pairs, bits, status);
  prof_mark(s, "k_fast_pairs");
  RST_CUDA(cudaGetLastError());
  if (labels_out)
    RST_CUDA(cudaMemcpyAsync(labels_out, uf, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  unsigned long long h[8];
  RST_TRY(fetch_u64(cnt, 8, h, s));
  out->T = (int64_t)(h[FC_R1] + h[FC_TREE]);
  out->pairs = pairs;
  out->bits = bits;
  out->nroots = (int64_t)h[FC_ROOTS];
  out->roots = roots;
  out->rounds = kSampleRounds;
  out->root_label = root >= 0 ? (int32_t)h[FC_ROOT_LABEL] : -1;
  set_stat(STAT_ROUNDS, out->rounds);
  set_stat(STAT_T, out->T);
  set_stat(STAT_NROOTS, out->nroots);
  return RST_OK;
}

template size_t ccfast_workspace_bytes<int32_t>(int64_t, int64_t);
template size_t ccfast_workspace_bytes<int64_t>(int64_t, int64_t);
template rst_status ccfast_run<int32_t>(Arena&, const int32_t*, const int32_t*, int64_t, int64_t, int32_t,
                                        int32_t*, CcOut*, cudaStream_t);
template rst_status ccfast_run<int64_t>(Arena&, const int64_t*, const int32_t*, int64_t, int64_t, int32_t,
                                        int32_t*, CcOut*, cudaStream_t);

}  // namespace rst
