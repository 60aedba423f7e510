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
