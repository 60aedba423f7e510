// Level-synchronous, direction-optimising BFS (Section III-A; the paper's
// baseline is Merrill et al.'s edge-centric BFS).  Parent rule: every vertex
// takes the minimum-id neighbour on the previous level, which makes the tree
// unique.
//
// Top-down steps expand the frontier queue.  When the graph's maximum degree
// is small every frontier vertex is one thread; otherwise the frontier's arcs
// are enumerated edge-centrically (a prefix sum of frontier degrees feeds the
// load-balanced merge-path walker, as in Merrill's expansion).  Newly reached
// vertices claim their level with atomicCAS and every frontier neighbour
// offers itself as parent with atomicMin.  Bottom-up steps (Beamer's
// direction optimisation) let each unvisited vertex scan its sorted row for
// the first neighbour on the current level, which is the minimum-id one.
//
// One kernel launch and one host read of the next frontier size per level:
// Theta(diameter) launches and synchronisations, the cost the paper
// attributes to BFS on high-diameter graphs.  Components that do not contain
// the root are searched afterwards from their minimum vertex id.
#include <climits>

#include "csr_walk.cuh"
#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

enum { BC_NEXT = 0, BC_MAXDEG = 1, BC_MINUNV = 2, BC_FEDGES = 3 };

template <class OffT>
__global__ void k_bfs_init(const OffT* __restrict__ off, int64_t n, int32_t* __restrict__ level,
                           int32_t* __restrict__ parent, unsigned long long* counters) {
  unsigned long long md = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
    md = d > md ? d : md;
    if (d == 0) {  // isolated: its own root at level 0
      level[v] = 0;
      parent[v] = (int32_t)v;
    } else {
      level[v] = -1;
      parent[v] = INT_MAX;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, md, d);
    md = o > md ? o : md;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(&counters[BC_MAXDEG], md);
}

__global__ void k_bfs_seed(int32_t src, int32_t* __restrict__ level, int32_t* __restrict__ parent,
                           int32_t* __restrict__ q) {
  level[src] = 0;
  parent[src] = src;
  q[0] = src;
}

// Several sources at once (one per graph of a disjoint union): each unvisited
// source starts at level 0; already-settled ones (isolated) are skipped.
__global__ void k_bfs_seed_many(const int32_t* __restrict__ seeds, int64_t ns, int32_t* __restrict__ level,
                                int32_t* __restrict__ parent, int32_t* __restrict__ q,
                                unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ns; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool fresh = false;
    int32_t s = -1;
    if (i < ns) {
      s = seeds[i];
      if (s >= 0) fresh = atomicCAS(&level[s], -1, 0) == -1;
      if (fresh) parent[s] = s;
    }
    const unsigned long long slot = block_reserve<kBlock>(&counters[BC_NEXT], fresh ? 1u : 0u);
    if (fresh) q[slot] = s;
  }
}

// Top-down, one thread per frontier vertex (small maximum degree).
template <class OffT>
__global__ void k_bfs_td_thread(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ q, int64_t nf, int32_t L,
                                int32_t* __restrict__ level, int32_t* __restrict__ parent,
                                int32_t* __restrict__ q2, unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nf; base += stride) {
    const int64_t i = base + threadIdx.x;
    int32_t u = -1;
    int64_t j = 0, hi = 0;
    if (i < nf) {
      u = q[i];
      j = (int64_t)off[u];
      hi = (int64_t)off[u + 1];
    }
    // every lane runs the same number of warp-collective appends
    int64_t mydeg = hi - j;
    int64_t maxdeg = mydeg;
    for (int d = 16; d > 0; d >>= 1) {
      const long long o = __shfl_xor_sync(0xffffffffu, (long long)maxdeg, d);
      maxdeg = o > maxdeg ? o : maxdeg;
    }
    for (int64_t k = 0; k < maxdeg; ++k) {
      bool fresh = false;
      int32_t v = 0;
      if (k < mydeg) {
        v = col[j + k];
        const int32_t old = atomicCAS(&level[v], -1, L + 1);
        if (old == -1 || old == L + 1) atomicMin(&parent[v], u);
        fresh = (old == -1);
      }
      const long long slot = warp_reserve(&counters[BC_NEXT], fresh);
      if (fresh) q2[slot] = v;
    }
  }
}

// Top-down, edge-centric over the frontier's arcs (virtual CSR fo over the queue).
template <class OffT>
struct TdEdgeFn {
  const OffT* __restrict__ off;
  const int32_t* __restrict__ col;
  const int32_t* __restrict__ q;
  const unsigned long long* __restrict__ fo;
  int32_t L;
  int32_t* __restrict__ level;
  int32_t* __restrict__ parent;
  int32_t* __restrict__ q2;
  unsigned long long* counter;
  __device__ __forceinline__ void end_tile() {}
  __device__ __forceinline__ void operator()(int, bool is_arc, int64_t row, int64_t arc) {
    bool fresh = false;
    int32_t v = 0;
    if (is_arc) {
      const int32_t u = q[row];
      v = col[(int64_t)off[u] + (arc - (int64_t)fo[row])];
      const int32_t old = atomicCAS(&level[v], -1, L + 1);
      if (old == -1 || old == L + 1) atomicMin(&parent[v], u);
      fresh = (old == -1);
    }
    const long long slot = warp_reserve(counter, fresh);
    if (fresh) q2[slot] = v;
  }
};

template <class OffT>
__global__ void __launch_bounds__(kMpThreads) k_bfs_td_edges(int64_t nf, int64_t fe, TdEdgeFn<OffT> f) {
  csr_for_each_arc<unsigned long long>(f.fo, nf, fe, f);
}

template <class OffT>
__global__ void k_bfs_fdeg(const OffT* __restrict__ off, const int32_t* __restrict__ q, int64_t nf,
                           unsigned long long* __restrict__ fdeg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = q[i];
    fdeg[i] = (unsigned long long)(off[u + 1] - off[u]);
  }
}

// Bottom-up: each unvisited vertex looks for its first neighbour on level L.
template <class OffT>
__global__ void k_bfs_bu(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t n, int32_t L,
                         int32_t* __restrict__ level, int32_t* __restrict__ parent, int32_t* __restrict__ q2,
                         unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    bool fresh = false;
    if (v < n && level[v] == -1) {
      const int64_t hi = (int64_t)off[v + 1];
      for (int64_t j = (int64_t)off[v]; j < hi; ++j) {
        const int32_t u = col[j];
        if (level[u] == L) {
          parent[v] = u;
          fresh = true;
          break;
        }
      }
    }
    const unsigned long long slot = block_reserve<kBlock>(&counters[BC_NEXT], fresh ? 1u : 0u);
    if (fresh) q2[slot] = (int32_t)v;
  }
}

// Levels of the bottom-up step are written after the step so that a vertex
// found at level L+1 is not mistaken for a level-L vertex within the step.
__global__ void k_bfs_commit(const int32_t* __restrict__ q2, int64_t nq, int32_t L, int32_t* __restrict__ level) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x)
    level[q2[i]] = L + 1;
}

__global__ void k_bfs_min_unvisited(int64_t n, const int32_t* __restrict__ level, unsigned long long* counters) {
  unsigned long long best = ~0ull;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (level[v] == -1) {
      best = (unsigned long long)v;
      break;  // grid-stride order: the first hit of each thread is its minimum
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, best, d);
    best = o < best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&counters[BC_MINUNV], best);
}

size_t bfs_workspace_bytes(int64_t n) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  return al(n * 4) * 3 + al((n + 1) * 8) + al(scan_tmp_words(n + 1) * 8);
}

static long long g_bfs_max_levels = 0;  // 0: unlimited (rst_set_option "bfs_max_levels")
void set_bfs_max_levels(long long v) { g_bfs_max_levels = v; }
long long get_bfs_max_levels() { return g_bfs_max_levels; }

// The search itself; buffers come from `ar` (sized by bfs_workspace_bytes).
// With a probe, only the root's search runs, for at most probe->max_levels
// levels, and the frontier size of every level is recorded.
template <class OffT>
static rst_status bfs_core(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                           const int32_t* seeds, int64_t nseeds, int32_t* parent, int32_t* level_out,
                           cudaStream_t s, BfsProbe* probe = nullptr) {
  DeviceState& st = state();
  int32_t* level = level_out ? level_out : ar.take<int32_t>(n);
  int32_t* qa = ar.take<int32_t>(n);
  int32_t* qb = ar.take<int32_t>(n);
  unsigned long long* fo = ar.take<unsigned long long>(n + 1);
  unsigned long long* tmp = ar.take<unsigned long long>(scan_tmp_words(n + 1));
  if (!level || !qa || !qb || !fo || !tmp) return RST_ERR_OOM;
  unsigned long long* cnt = dev_counter(0);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  const int gN = grid_for(n);
  RST_LAUNCH(k_bfs_init<OffT>, gN, kBlock, 0, s)(off, n, level, parent, cnt);
  unsigned long long h[8];
  RST_TRY(fetch_u64(cnt, 8, h, s));
  const int64_t maxdeg = (int64_t)h[BC_MAXDEG];
  const bool thread_td = maxdeg <= 64;
  int32_t src = seeds ? -2 : root;  // -2: the multi-source first search
  int64_t levels_total = 0;
  while (src >= 0 || src == -2) {
    int32_t probe_level = -1;
    int64_t nf = 1;
    if (src == -2) {
      RST_CUDA(cudaMemsetAsync(&cnt[BC_NEXT], 0, sizeof(unsigned long long), s));
      RST_LAUNCH(k_bfs_seed_many, grid_for(nseeds), kBlock, 0, s)(seeds, nseeds, level, parent, qa, cnt);
      RST_TRY(fetch_u64(&cnt[BC_NEXT], 1, h, s));
      nf = (int64_t)h[0];
    } else {
      RST_CUDA(cudaMemcpyAsync(st.hostbuf, level + src, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RST_CUDA(cudaStreamSynchronize(s));
      std::memcpy(&probe_level, st.hostbuf, sizeof(int32_t));
      if (probe_level == -1) RST_LAUNCH(k_bfs_seed, 1, 1, 0, s)(src, level, parent, qa);
    }
    if (probe_level == -1 && nf > 0) {
      int32_t L = 0;
      bool bottom_up = false;
      int32_t* q = qa;
      int32_t* q2 = qb;
      while (nf > 0) {
        if (probe) {
          if (L < BfsProbe::kMax) probe->frontier[L] = nf;
          probe->reached += nf;
          probe->levels = L + 1;
          if (L + 1 >= probe->max_levels) break;
        }
        if (!probe && g_bfs_max_levels > 0 && L >= g_bfs_max_levels) return RST_ERR_NOT_CONVERGED;
        RST_CUDA(cudaMemsetAsync(&cnt[BC_NEXT], 0, sizeof(unsigned long long), s));
        const bool want_bu = nf > n / tuning().bfs_bu_div;
        if (want_bu) {
          RST_LAUNCH(k_bfs_bu<OffT>, gN, kBlock, 0, s)(off, col, n, L, level, parent, q2, cnt);
        } else if (thread_td) {
          RST_LAUNCH(k_bfs_td_thread<OffT>, grid_for(nf), kBlock, 0, s)(off, col, q, nf, L, level, parent, q2, cnt);
        } else {
          RST_LAUNCH(k_bfs_fdeg<OffT>, grid_for(nf), kBlock, 0, s)(off, q, nf, fo);
          RST_TRY(scan_exclusive_u64(fo, fo, nf, tmp, s));
          RST_CUDA(cudaMemcpyAsync(&cnt[BC_FEDGES], fo + nf, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToDevice, s));
          RST_TRY(fetch_u64(&cnt[BC_FEDGES], 1, h, s));
          const int64_t fe = (int64_t)h[0];
          TdEdgeFn<OffT> f{off, col, q, fo, L, level, parent, q2, &cnt[BC_NEXT]};
          const int64_t tiles = (nf + fe + kMpTile - 1) / kMpTile;
          const int g = (int)(tiles < (int64_t)device_info().sms * 8 ? (tiles > 0 ? tiles : 1)
                                                                      : (int64_t)device_info().sms * 8);
          RST_LAUNCH(k_bfs_td_edges<OffT>, g, kMpThreads, 0, s)(nf, fe, f);
        }
        RST_CUDA(cudaGetLastError());
        RST_TRY(fetch_u64(&cnt[BC_NEXT], 1, h, s));
        const int64_t nn = (int64_t)h[0];
        if (want_bu && nn > 0) RST_LAUNCH(k_bfs_commit, grid_for(nn), kBlock, 0, s)(q2, nn, L, level);
        bottom_up = want_bu;
        std::swap(q, q2);
        nf = nn;
        ++L;
        if (L > n + 1) return RST_ERR_NOT_CONVERGED;
      }
      (void)bottom_up;
      levels_total += L;
      if (probe) {
        probe->finished = (nf == 0);
        probe->last_frontier = nf;
        break;
      }
    }
    if (probe) break;  // the probe only searches the root's component
    // next component: minimum unvisited vertex
    RST_CUDA(cudaMemsetAsync(&cnt[BC_MINUNV], 0xff, sizeof(unsigned long long), s));
    RST_LAUNCH(k_bfs_min_unvisited, gN, kBlock, 0, s)(n, level, cnt);
    RST_CUDA(cudaGetLastError());
    RST_TRY(fetch_u64(&cnt[BC_MINUNV], 1, h, s));
    src = h[0] == ~0ull ? -1 : (int32_t)h[0];
  }
  set_stat(STAT_LEVELS, levels_total);
  return RST_OK;
}

template <class OffT>
static rst_status bfs_impl(const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                           int32_t* parent, int32_t* level_out, cudaStream_t s) {
  RST_TRY(ensure_workspace(bfs_workspace_bytes(n)));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  RST_TRY(bfs_core<OffT>(ar, off, col, n, A, root, nullptr, 0, parent, level_out, s));
  return read_device_error(s);
}

rst_status run_bfs(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                   int32_t root, int32_t* parent, int32_t* level_out, cudaStream_t s) {
  if (offsets_bits == 32) return bfs_impl<int32_t>((const int32_t*)off, cols, n, m, root, parent, level_out, s);
  return bfs_impl<int64_t>((const int64_t*)off, cols, n, m, root, parent, level_out, s);
}

// ------------------------------------------------------------------ device-driven BFS
//
// The same search (same levels, same minimum-id parents, leftover components
// from their minimum vertex) with the level loop on the device: the body of a
// CUDA-graph while node is one kernel per level, and the last block of each
// launch decides the next step (top-down, bottom-up, or the seek for the next
// component's minimum vertex) and sets the loop condition.  No host
// synchronisation per level.
//
// Top-down expansion gathers Merrill-style in three tiers: rows of up to 32
// arcs are walked by their own thread, rows of up to one block by a warp,
// longer rows by the whole block; rows longer than kBigDeg are queued apart
// when discovered and expanded by several blocks (a group of kGroupBlocks per
// row, the whole grid for rows of kHugeDeg or more).  Frontier entries carry
// the row start and degree read when the vertex was discovered, so the next
// level reads no offsets.

constexpr uint32_t kBigDeg = 4096;
constexpr uint32_t kHugeDeg = 1u << 18;
constexpr int kGroupBlocks = 16;
constexpr unsigned long long kSeekWindow0 = 1ull << 16;

struct __align__(16) FEntry {
  int32_t v;
  uint32_t deg;
  int64_t start;
};

enum { BD_TD = 0, BD_BU = 1, BD_SEEK = 2, BD_DONE = 3 };

// Fields that many blocks update or poll at once sit on their own 128-byte
// lines, apart from the step description every block reads.
struct BfsDevCtl {
  int L;     // level of the frontier being expanded
  int mode;  // BD_*
  int par;   // parity of the frontier queues
  int bu_div;
  long long cap;                 // level cap (0: none)
  unsigned long long max_iters;  // bound on loop iterations
  unsigned long long nf;         // frontier entries (short rows)
  unsigned long long nbig;       // frontier entries (long rows)
  unsigned long long cursor;     // every vertex below it is visited
  unsigned long long window;     // seek window length
  unsigned long long iters;      // loop iterations so far
  unsigned long long levels;     // levels expanded over all searches
  alignas(128) unsigned long long nn;  // next frontier, short rows (append counter)
  alignas(128) unsigned long long nbn;       // next frontier, long rows (append counter)
  unsigned long long seek_min;               // smallest unvisited vertex found by a seek
  alignas(128) unsigned int done;            // blocks of the current launch that finished
  alignas(128) unsigned int arrive;          // persistent variant: blocks at the level barrier
  alignas(128) unsigned int gen;             // persistent variant: barrier generation
};

// The fields one launch reads (a register copy of the control block).
struct BfsStep {
  int L, mode, par;
  unsigned long long nf, nbig, cursor, window;
};

template <class OffT>
struct BfsDevArgs {
  const OffT* off;
  const int32_t* col;
  int64_t n;
  int32_t* level;
  int32_t* parent;
  FEntry* q[2];
  FEntry* big[2];
  int64_t bigcap;
  BfsDevCtl* ctl;
  uint32_t* status;
};

// Visit arc u -> v of a top-down step (valid lanes only) and append v to the
// next frontier when this arc reached it first.  Warp-collective: every lane
// of the warp calls it.
template <class OffT>
__device__ __forceinline__ void bfsd_visit(const BfsDevArgs<OffT>& a, int32_t L, int nxt, bool valid,
                                           int32_t v, int32_t u) {
  bool fresh = false;
  int64_t vs = 0;
  uint32_t vd = 0;
  if (valid) {
    if (v < 0 || (int64_t)v >= a.n) {
      raise_error(a.status, DERR_INDEX);
    } else {
      const int32_t old = atomicCAS(&a.level[v], -1, L + 1);
      if (old == -1 || old == L + 1) atomicMin(&a.parent[v], u);
      fresh = old == -1;
      if (fresh) {
        vs = (int64_t)a.off[v];
        vd = (uint32_t)((int64_t)a.off[v + 1] - vs);
      }
    }
  }
  const bool big = fresh && vd > kBigDeg;
  const bool norm = fresh && !big;
  const long long slot = warp_reserve(&a.ctl->nn, norm);
  if (norm) {
    FEntry e;
    e.v = v;
    e.deg = vd;
    e.start = vs;
    a.q[nxt][slot] = e;
  }
  if (big) {
    const unsigned long long b = atomicAdd(&a.ctl->nbn, 1ull);
    if ((int64_t)b < a.bigcap) {
      FEntry e;
      e.v = v;
      e.deg = vd;
      e.start = vs;
      a.big[nxt][b] = e;
    } else {
      raise_error(a.status, DERR_CAPACITY);
    }
  }
}

// Up to kTdBatch arcs u -> col[j0 + k], k < cnt (cnt may be <= 0: no arcs):
// the column loads, then the level claims, then the discovered vertices' row
// bounds are issued together, and the warp reserves its queue slots once.
// Warp-collective.
constexpr int kTdBatch = 4;
template <class OffT>
__device__ __forceinline__ void bfsd_visit_batch(const BfsDevArgs<OffT>& a, int32_t L, int nxt, int32_t u,
                                                 int64_t j0, int cnt) {
  int32_t v[kTdBatch];
  int32_t old[kTdBatch];
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k) v[k] = k < cnt ? a.col[j0 + k] : -1;
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k) {
    old[k] = 0;
    if (k < cnt) {
      if (v[k] < 0 || (int64_t)v[k] >= a.n) {
        raise_error(a.status, DERR_INDEX);
        v[k] = -1;
      } else {
        old[k] = atomicCAS(&a.level[v[k]], -1, L + 1);
      }
    }
  }
  unsigned fresh = 0;
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k)
    if (k < cnt && v[k] >= 0) {
      if (old[k] == -1 || old[k] == L + 1) atomicMin(&a.parent[v[k]], u);
      if (old[k] == -1) fresh |= 1u << k;
    }
  int64_t vs[kTdBatch];
  int64_t ve[kTdBatch];
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k) {
    vs[k] = 0;
    ve[k] = 0;
    if ((fresh >> k) & 1u) {
      vs[k] = (int64_t)a.off[v[k]];
      ve[k] = (int64_t)a.off[v[k] + 1];
    }
  }
  unsigned norm = 0;
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k)
    if (((fresh >> k) & 1u) && ve[k] - vs[k] <= (int64_t)kBigDeg) norm |= 1u << k;
  // one reservation per warp for every lane's short rows
  const unsigned mine = (unsigned)__popc(norm);
  const int lane = threadIdx.x & 31;
  unsigned x = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  const unsigned total = __shfl_sync(0xffffffffu, x, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(&a.ctl->nn, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31) + (x - mine);
#pragma unroll
  for (int k = 0; k < kTdBatch; ++k) {
    if (!((fresh >> k) & 1u)) continue;
    FEntry e;
    e.v = v[k];
    e.deg = (uint32_t)(ve[k] - vs[k]);
    e.start = vs[k];
    if ((norm >> k) & 1u) {
      a.q[nxt][base++] = e;
    } else {
      const unsigned long long b = atomicAdd(&a.ctl->nbn, 1ull);
      if ((int64_t)b < a.bigcap)
        a.big[nxt][b] = e;
      else
        raise_error(a.status, DERR_CAPACITY);
    }
  }
}

template <class OffT>
__device__ __forceinline__ void bfsd_top_down(const BfsDevArgs<OffT>& a, const BfsStep& c) {
  __shared__ FEntry s_e[kBlock];
  __shared__ int s_owner;
  __shared__ int32_t s_u;
  __shared__ int64_t s_j, s_hi;
  const int32_t L = c.L;
  const int par = c.par, nxt = par ^ 1;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // long rows: loaded a block's worth at a time; a row of kHugeDeg or more is
  // walked by the whole grid, any other by one group of kGroupBlocks blocks
  const int64_t nbig = (int64_t)c.nbig;
  const FEntry* __restrict__ bq = a.big[par];
  const int groups = gridDim.x >= kGroupBlocks ? (int)(gridDim.x / kGroupBlocks) : 1;
  const int gsize = gridDim.x >= kGroupBlocks ? kGroupBlocks : (int)gridDim.x;
  const int my_group = (int)(blockIdx.x / gsize);
  const int64_t gstride = (int64_t)gsize * blockDim.x;
  for (int64_t b0 = 0; b0 < nbig; b0 += blockDim.x) {
    if (b0 + threadIdx.x < nbig) s_e[threadIdx.x] = bq[b0 + threadIdx.x];
    __syncthreads();
    const int cnt = (int)(nbig - b0 < (int64_t)blockDim.x ? nbig - b0 : (int64_t)blockDim.x);
    for (int r = 0; r < cnt; ++r) {
      const FEntry e = s_e[r];
      int64_t first, step;
      if (e.deg >= kHugeDeg) {
        first = (int64_t)blockIdx.x * blockDim.x;
        step = stride;
      } else if ((int)((b0 + r) % groups) == my_group && my_group < groups) {
        first = (int64_t)(blockIdx.x - (unsigned)my_group * gsize) * blockDim.x;
        step = gstride;
      } else {
        continue;
      }
      for (int64_t k0 = first + (threadIdx.x & ~31); k0 < (int64_t)e.deg; k0 += step) {
        const int64_t k = k0 + lane;
        const bool valid = k < (int64_t)e.deg;
        bfsd_visit(a, L, nxt, valid, valid ? a.col[e.start + k] : 0, e.v);
      }
    }
    __syncthreads();
  }
  // short rows: thread, warp and block tiers
  const int64_t nf = (int64_t)c.nf;
  const FEntry* __restrict__ q = a.q[par];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nf; base += stride) {
    const int64_t i = base + threadIdx.x;
    int32_t u = -1;
    int64_t j = 0, hi = 0;
    if (i < nf) {
      const FEntry e = q[i];
      u = e.v;
      j = e.start;
      hi = e.start + (int64_t)e.deg;
    }
    while (true) {  // block tier: rows longer than a block
      if (threadIdx.x == 0) s_owner = -1;
      __syncthreads();
      if (hi - j > (int64_t)blockDim.x) s_owner = (int)threadIdx.x;
      __syncthreads();
      const int owner = s_owner;
      if (owner < 0) break;
      if ((int)threadIdx.x == owner) {
        s_u = u;
        s_j = j;
        s_hi = hi;
        j = hi;
      }
      __syncthreads();
      const int32_t cu = s_u;
      const int64_t cj = s_j, chi = s_hi;
      for (int64_t k0 = cj; k0 < chi; k0 += blockDim.x) {
        const int64_t k = k0 + threadIdx.x;
        const bool valid = k < chi;
        bfsd_visit(a, L, nxt, valid, valid ? a.col[k] : 0, cu);
      }
      __syncthreads();
    }
    while (true) {  // warp tier: rows longer than 32 arcs
      const unsigned m = __ballot_sync(0xffffffffu, hi - j > 32);
      if (!m) break;
      const int leader = __ffs(m) - 1;
      const int32_t wu = __shfl_sync(0xffffffffu, u, leader);
      const int64_t wj = __shfl_sync(0xffffffffu, j, leader);
      const int64_t whi = __shfl_sync(0xffffffffu, hi, leader);
      if (lane == leader) j = hi;
      for (int64_t k0 = wj; k0 < whi; k0 += 32) {
        const int64_t k = k0 + lane;
        const bool valid = k < whi;
        bfsd_visit(a, L, nxt, valid, valid ? a.col[k] : 0, wu);
      }
    }
    // thread tier: at most 32 arcs each, kTdBatch at a time with all their
    // loads and atomics in flight together
    const int rem = (int)(hi - j);
    int mx = rem;
    for (int d = 16; d > 0; d >>= 1) {
      const int o = __shfl_xor_sync(0xffffffffu, mx, d);
      mx = o > mx ? o : mx;
    }
    for (int t0 = 0; t0 < mx; t0 += kTdBatch) bfsd_visit_batch(a, L, nxt, u, j + t0, rem - t0);
  }
}

// Bottom-up: each unvisited vertex takes the first neighbour of its sorted
// row on level L (the minimum-id one).  Its level is written at once: L + 1
// is never mistaken for L by a neighbour in the same step.
template <class OffT>
__device__ __forceinline__ void bfsd_bottom_up(const BfsDevArgs<OffT>& a, const BfsStep& c) {
  const int32_t L = c.L;
  const int nxt = c.par ^ 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
    const int64_t v = base + threadIdx.x;
    bool fresh = false;
    int64_t lo = 0, hi = 0;
    if (v < a.n && a.level[v] == -1) {
      lo = (int64_t)a.off[v];
      hi = (int64_t)a.off[v + 1];
      for (int64_t j = lo; j < hi; ++j) {
        const int32_t u = a.col[j];
        if (u < 0 || (int64_t)u >= a.n) {
          raise_error(a.status, DERR_INDEX);
          break;
        }
        if (a.level[u] == L) {
          a.parent[v] = u;
          a.level[v] = L + 1;
          fresh = true;
          break;
        }
      }
    }
    const uint32_t deg = (uint32_t)(hi - lo);
    const bool big = fresh && deg > kBigDeg;
    const bool norm = fresh && !big;
    const long long slot = warp_reserve(&a.ctl->nn, norm);
    FEntry e;
    e.v = (int32_t)v;
    e.deg = deg;
    e.start = lo;
    if (norm) a.q[nxt][slot] = e;
    if (big) {
      const unsigned long long b = atomicAdd(&a.ctl->nbn, 1ull);
      if ((int64_t)b < a.bigcap)
        a.big[nxt][b] = e;
      else
        raise_error(a.status, DERR_CAPACITY);
    }
  }
}

// The smallest unvisited vertex in the current seek window.
template <class OffT>
__device__ __forceinline__ void bfsd_seek(const BfsDevArgs<OffT>& a, const BfsStep& c) {
  const int64_t lo = (int64_t)c.cursor;
  const int64_t hi = lo + (int64_t)c.window < a.n ? lo + (int64_t)c.window : a.n;
  unsigned long long best = ~0ull;
  for (int64_t v = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < hi;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (a.level[v] == -1) {
      best = (unsigned long long)v;
      break;  // grid-stride order: a thread's first hit is its smallest
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, best, d);
    best = o < best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&a.ctl->seek_min, best);
}

// Starts the search at `src` (a vertex with edges, level already -1 or set).
template <class OffT>
__device__ void bfsd_seed(const BfsDevArgs<OffT>& a, BfsDevCtl* c, int32_t src) {
  a.level[src] = 0;
  a.parent[src] = src;
  FEntry e;
  e.v = src;
  e.start = (int64_t)a.off[src];
  e.deg = (uint32_t)((int64_t)a.off[src + 1] - e.start);
  c->L = 0;
  if (e.deg > kBigDeg) {
    a.big[c->par][0] = e;
    c->nbig = 1;
    c->nf = 0;
  } else {
    a.q[c->par][0] = e;
    c->nf = 1;
    c->nbig = 0;
  }
  c->mode = (1 > a.n / c->bu_div) ? BD_BU : BD_TD;
}

template <class OffT>
__global__ void k_bfsd_start(BfsDevArgs<OffT> a, int32_t root, int bu_div, long long cap,
                             unsigned long long max_iters) {
  BfsDevCtl* c = a.ctl;
  c->par = 0;
  c->bu_div = bu_div;
  c->cap = cap;
  c->max_iters = max_iters;
  c->nn = c->nbn = 0;
  c->cursor = 0;
  c->window = kSeekWindow0;
  c->seek_min = ~0ull;
  c->iters = 0;
  c->levels = 0;
  c->done = 0;
  c->arrive = 0;
  c->gen = 0;
  c->nf = c->nbig = 0;
  c->L = 0;
  if (a.off[root + 1] - a.off[root] > 0) {
    bfsd_seed(a, c, root);
  } else {
    c->mode = BD_SEEK;  // an isolated root is already its own tree
  }
}

// After a launch (one thread): the next step and the loop condition.
template <class OffT, bool kGraph>
__device__ void bfsd_finish(const BfsDevArgs<OffT>& a, cudaGraphConditionalHandle h, int use_handle) {
  BfsDevCtl* c = a.ctl;
  const int mode = c->mode;
  bool more = true;
  c->iters += 1;
  if (mode == BD_TD || mode == BD_BU) {
    c->levels += 1;
    const unsigned long long nn = c->nn, nb = c->nbn;
    if (nn + nb > 0) {
      const int L2 = c->L + 1;
      if (c->cap > 0 && (long long)L2 >= c->cap) {
        raise_error(a.status, DERR_ROUND_LIMIT);
        more = false;
      }
      c->L = L2;
      c->par ^= 1;
      c->nf = nn;
      c->nbig = nb;
      c->mode = ((long long)(nn + nb) > a.n / c->bu_div) ? BD_BU : BD_TD;
    } else {
      c->nf = c->nbig = 0;
      c->window = kSeekWindow0;
      c->mode = BD_SEEK;
    }
  } else if (mode == BD_SEEK) {
    const unsigned long long m = c->seek_min;
    if (m != ~0ull) {
      bfsd_seed(a, c, (int32_t)m);
      c->cursor = m + 1;
    } else {
      c->cursor += c->window;
      c->window = c->window * 2 < (unsigned long long)a.n ? c->window * 2 : (unsigned long long)a.n;
      if (c->cursor >= (unsigned long long)a.n) {
        c->mode = BD_DONE;
        more = false;
      }
    }
  } else {
    more = false;
  }
  if (c->iters >= c->max_iters && more) {
    raise_error(a.status, DERR_ROUND_LIMIT);
    more = false;
  }
  c->nn = 0;
  c->nbn = 0;
  c->seek_min = ~0ull;
  c->done = 0;
  if (!more) c->mode = BD_DONE;
  if constexpr (kGraph) {
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

template <class OffT>
__global__ void __launch_bounds__(kBlock) k_bfsd_step(BfsDevArgs<OffT> a, cudaGraphConditionalHandle h,
                                                      int use_handle) {
  // the step's fields, read before any block can finish the launch
  BfsStep c;
  c.mode = a.ctl->mode;
  c.L = a.ctl->L;
  c.par = a.ctl->par;
  c.nf = a.ctl->nf;
  c.nbig = a.ctl->nbig;
  c.cursor = a.ctl->cursor;
  c.window = a.ctl->window;
  if (c.mode == BD_TD)
    bfsd_top_down(a, c);
  else if (c.mode == BD_BU)
    bfsd_bottom_up(a, c);
  else if (c.mode == BD_SEEK)
    bfsd_seek(a, c);
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&a.ctl->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    bfsd_finish<OffT, true>(a, h, use_handle);
  }
}

// Persistent variant: one cooperative launch (every block resident) runs all
// levels.  Blocks meet at a grid barrier after each level; the last block to
// arrive decides the next step and releases the others by advancing the
// barrier generation.  Every wait is bounded: a block that waits longer than
// kBarrierSpins polls gives up, sets DERR_ROUND_LIMIT and leaves, and so do
// the others in turn.
constexpr unsigned long long kBarrierSpins = 1ull << 25;

template <class OffT>
__global__ void __launch_bounds__(kBlock) k_bfsp(BfsDevArgs<OffT> a) {
  __shared__ int s_stop;
  BfsDevCtl* ctl = a.ctl;
  for (;;) {
    BfsStep c;
    c.mode = *(volatile int*)&ctl->mode;
    c.L = *(volatile int*)&ctl->L;
    c.par = *(volatile int*)&ctl->par;
    c.nf = *(volatile unsigned long long*)&ctl->nf;
    c.nbig = *(volatile unsigned long long*)&ctl->nbig;
    c.cursor = *(volatile unsigned long long*)&ctl->cursor;
    c.window = *(volatile unsigned long long*)&ctl->window;
    if (c.mode == BD_DONE) break;
    if (c.mode == BD_TD)
      bfsd_top_down(a, c);
    else if (c.mode == BD_BU)
      bfsd_bottom_up(a, c);
    else
      bfsd_seek(a, c);
    __syncthreads();
    if (threadIdx.x == 0) {
      s_stop = 0;
      const unsigned int gen = *(volatile unsigned int*)&ctl->gen;
      __threadfence();
      if (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1) {
        __threadfence();
        ctl->arrive = 0;
        bfsd_finish<OffT, false>(a, cudaGraphConditionalHandle{}, 0);
        __threadfence();
        atomicAdd(&ctl->gen, 1u);  // release
      } else {
        unsigned long long spins = 0;
        while (*(volatile unsigned int*)&ctl->gen == gen) {
          if (++spins > kBarrierSpins) {
            raise_error(a.status, DERR_ROUND_LIMIT);
            s_stop = 1;
            break;
          }
          __nanosleep(64);
        }
        __threadfence();
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
}

static int bfsd_grid() { return device_info().sms * tuning().bfsd_bps; }

size_t bfs_device_workspace_bytes(int64_t n, int64_t A) {
  Arena a;
  a.counting = true;
  a.take<int32_t>(n);
  a.take<FEntry>(n + 1);
  a.take<FEntry>(n + 1);
  a.take<FEntry>(A / kBigDeg + 2);
  a.take<FEntry>(A / kBigDeg + 2);
  a.take<BfsDevCtl>(1);
  return a.used;
}

// One instantiated while-loop graph per binding of buffers and grid.
struct BfsGraph {
  bool valid = false;
  const void* key_off = nullptr;
  const void* key_col = nullptr;
  const void* key_ctl = nullptr;
  const void* key_parent = nullptr;
  const void* key_level = nullptr;
  int64_t key_n = 0;
  int key_dev = -1, key_grid = 0;
  cudaGraphExec_t exec = nullptr;
};
constexpr int kBfsGraphCache = 4;
static BfsGraph g_bfs_graphs[kBfsGraphCache];
static int g_bfs_graph_next = 0;
static cudaStream_t g_bfs_capture[64] = {};

void destroy_bfs_graphs() {
  for (auto& g : g_bfs_graphs) {
    if (g.valid && g.exec) cudaGraphExecDestroy(g.exec);
    g = BfsGraph{};
  }
}

template <class OffT>
static rst_status bfsd_graph_for(const BfsDevArgs<OffT>& a, cudaGraphExec_t* out) {
  int dev = 0;
  RST_CUDA(cudaGetDevice(&dev));
  const int grid = bfsd_grid();
  for (auto& g : g_bfs_graphs)
    if (g.valid && g.key_off == a.off && g.key_col == a.col && g.key_ctl == a.ctl &&
        g.key_parent == a.parent && g.key_level == a.level && g.key_n == a.n && g.key_dev == dev &&
        g.key_grid == grid) {
      *out = g.exec;
      return RST_OK;
    }
  if (dev < 0 || dev >= 64) return RST_ERR_UNSUPPORTED;
  if (!g_bfs_capture[dev]) RST_CUDA(cudaStreamCreateWithFlags(&g_bfs_capture[dev], cudaStreamNonBlocking));
  cudaStream_t cs = g_bfs_capture[dev];
  cudaGraph_t graph = nullptr;
  RST_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  RST_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  RST_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  RST_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  k_bfsd_step<OffT><<<grid, kBlock, 0, cs>>>(a, h, 1);
  cudaGraph_t captured = nullptr;
  RST_CUDA(cudaStreamEndCapture(cs, &captured));
  cudaGraphExec_t exec = nullptr;
  RST_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  RST_CUDA(cudaGraphDestroy(graph));
  BfsGraph& slot = g_bfs_graphs[g_bfs_graph_next];
  g_bfs_graph_next = (g_bfs_graph_next + 1) % kBfsGraphCache;
  if (slot.valid && slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.valid = true;
  slot.key_off = a.off;
  slot.key_col = a.col;
  slot.key_ctl = a.ctl;
  slot.key_parent = a.parent;
  slot.key_level = a.level;
  slot.key_n = a.n;
  slot.key_dev = dev;
  slot.key_grid = grid;
  slot.exec = exec;
  *out = exec;
  return RST_OK;
}

// Grid of the persistent variant: as many resident blocks as fit (capped by
// the tuning knob), so that a cooperative launch can hold them all.
template <class OffT>
static rst_status bfsp_grid(int* grid) {
  int per_sm = 0;
  RST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfsp<OffT>, kBlock, 0));
  if (per_sm < 1) return RST_ERR_UNSUPPORTED;
  const int want = tuning().bfsp_bps;
  *grid = device_info().sms * (per_sm < want ? per_sm : want);
  return RST_OK;
}

template <class OffT>
static rst_status bfs_device_impl(const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                                  int32_t* parent, int32_t* level_out, cudaStream_t s, bool persistent) {
  RST_TRY(ensure_workspace(bfs_device_workspace_bytes(n, A)));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  BfsDevArgs<OffT> a;
  a.off = off;
  a.col = col;
  a.n = n;
  int32_t* lv = ar.take<int32_t>(n);
  a.level = level_out ? level_out : lv;
  a.parent = parent;
  a.q[0] = ar.take<FEntry>(n + 1);
  a.q[1] = ar.take<FEntry>(n + 1);
  a.bigcap = A / kBigDeg + 2;
  a.big[0] = ar.take<FEntry>(a.bigcap);
  a.big[1] = ar.take<FEntry>(a.bigcap);
  a.ctl = ar.take<BfsDevCtl>(1);
  a.status = st.status;
  if (ar.used > ar.cap) return RST_ERR_OOM;
  unsigned long long* cnt = dev_counter(0);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  RST_LAUNCH(k_bfs_init<OffT>, grid_for(n), kBlock, 0, s)(off, n, a.level, parent, cnt);
  const unsigned long long max_iters = 4ull * (unsigned long long)n + 1024;
  RST_LAUNCH(k_bfsd_start<OffT>, 1, 1, 0, s)(a, root, tuning().bfs_bu_div, g_bfs_max_levels, max_iters);
  static const bool eager = getenv("RST_EAGER") != nullptr;
  if (persistent) {
    int grid = 0;
    RST_TRY(bfsp_grid<OffT>(&grid));
    void* params[] = {&a};
    count_launch();
    RST_CUDA(cudaLaunchCooperativeKernel((const void*)k_bfsp<OffT>, dim3(grid), dim3(kBlock), params, 0, s));
  } else if (!eager) {
    cudaGraphExec_t exec = nullptr;
    RST_TRY(bfsd_graph_for<OffT>(a, &exec));
    RST_CUDA(cudaGraphLaunch(exec, s));
  } else {
    for (unsigned long long it = 0; it < max_iters + 1; ++it) {
      RST_LAUNCH(k_bfsd_step<OffT>, bfsd_grid(), kBlock, 0, s)(a, cudaGraphConditionalHandle{}, 0);
      RST_CUDA(cudaGetLastError());
      unsigned long long w = 0;
      RST_TRY(fetch_u64(reinterpret_cast<const unsigned long long*>(&a.ctl->L), 1, &w, s));
      if ((int)(w >> 32) == BD_DONE) break;  // {L, mode} read as one word
    }
  }
  RST_CUDA(cudaGetLastError());
  unsigned long long h[2];
  RST_TRY(fetch_u64(&a.ctl->iters, 2, h, s));
  if (!eager && !persistent) count_launches((long long)h[0]);
  set_stat(STAT_LEVELS, (long long)h[1]);
  return read_device_error(s);
}

rst_status run_bfs_device(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                          int32_t root, int32_t* parent, int32_t* level_out, cudaStream_t s, bool persistent) {
  if (offsets_bits == 32)
    return bfs_device_impl<int32_t>((const int32_t*)off, cols, n, m, root, parent, level_out, s, persistent);
  return bfs_device_impl<int64_t>((const int64_t*)off, cols, n, m, root, parent, level_out, s, persistent);
}

rst_status bfs_probe_in(Arena& ar, const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                        int32_t root, int32_t* parent_scratch, BfsProbe* probe, cudaStream_t s) {
  if (offsets_bits == 32)
    return bfs_core<int32_t>(ar, (const int32_t*)off, cols, n, m, root, nullptr, 0, parent_scratch, nullptr, s, probe);
  return bfs_core<int64_t>(ar, (const int64_t*)off, cols, n, m, root, nullptr, 0, parent_scratch, nullptr, s, probe);
}

rst_status bfs_multi_in(Arena& ar, const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                        const int32_t* seeds, int64_t nseeds, int32_t* parent, cudaStream_t s) {
  if (offsets_bits == 32)
    return bfs_core<int32_t>(ar, (const int32_t*)off, cols, n, m, -1, seeds, nseeds, parent, nullptr, s);
  return bfs_core<int64_t>(ar, (const int64_t*)off, cols, n, m, -1, seeds, nseeds, parent, nullptr, s);
}

}  // namespace rst
