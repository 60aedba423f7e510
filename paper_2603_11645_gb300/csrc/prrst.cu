// Path-reversal rooted spanning tree, PR-RST (Section III-C).
//
// A rooted forest P (every vertex its own tree at the start) is grown by
// rounds of hooking that alternate a minimum and a maximum rule: an arc (u,v)
// whose trees have roots ru != rv is eligible for tree ru when rv < ru
// (minimum rule, even rounds) or rv > ru (maximum rule, odd rounds), so the
// hooks of a round never form a cycle; each tree takes its eligible arc with
// the smallest key (u << 32 | v) by one 64-bit atomicMin.  A hooking tree is
// re-rooted at u by reversing the tree path u -> root and grafted under v.
//
// The path is found with the special ancestors of the paper: pointer jumping
// keeps its history anc[k][x] = 2^k-th ancestor of x (anc[0] = P), and the
// marks spread from u over the levels k = K-1 .. 0 (x marked => anc[k][x]
// marked), which reaches every ancestor of u in K passes.  Reversal is one
// data-parallel pass: every marked x sets Q[P[x]] = x, the bottom vertex u
// takes Q[u] = v, all other vertices keep P.  The last round has no hook.
// Finally each tree is re-rooted at the requested root (its tree) or at its
// minimum vertex id, with the same mark-and-reverse step.
#include <climits>

#include "csr_walk.cuh"
#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

namespace {

constexpr int kPrMaxLevels = 32;
constexpr int kPrMaxRounds = 256;

__global__ void k_pr_iota(int64_t n, int32_t* __restrict__ P) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    P[v] = (int32_t)v;
}

// One pointer-jumping step with history: up[x] = low[low[x]]; flags a change.
__global__ void k_pr_jump(int64_t n, const int32_t* __restrict__ low, int32_t* __restrict__ up, int32_t* changed) {
  bool ch = false;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = low[x];
    const int32_t b = low[a];
    up[x] = b;
    ch = ch || (b != a);
  }
  if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) *changed = 1;
}

// Several doubling levels per launch (the paper's several pointer jumps per
// global synchronisation): level k+i of x is computed from level k alone, by
// recomputing the intermediate ancestors it needs (2^i dependent reads), so
// every level written is exactly the 2^(k+i)-th ancestor.  changed[i-1] is
// set when level k+i differs from level k+i-1 somewhere.
constexpr int kPrMaxPerLaunch = 3;
__global__ void k_pr_jump_multi(int64_t n, const int32_t* __restrict__ low, int32_t* __restrict__ up1,
                                int32_t* __restrict__ up2, int32_t* __restrict__ up3, int levels,
                                int32_t* changed);
__global__ void k_pr_jump_multi(int64_t n, const int32_t* __restrict__ low, int32_t* __restrict__ up1,
                                int32_t* __restrict__ up2, int32_t* __restrict__ up3, int levels,
                                int32_t* changed) {
  bool ch[kPrMaxPerLaunch] = {false, false, false};
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a0 = low[x];
    const int32_t a1 = low[a0];
    up1[x] = a1;
    ch[0] = ch[0] || (a1 != a0);
    if (levels >= 2) {
      // level k+2 of x = level k+1 of a1 = two level-k steps from a1
      const int32_t a2 = low[low[a1]];
      up2[x] = a2;
      ch[1] = ch[1] || (a2 != a1);
      if (levels >= 3) {
        // level k+3 of x = level k+2 of a2 = four level-k steps from a2
        const int32_t a3 = low[low[low[low[a2]]]];
        up3[x] = a3;
        ch[2] = ch[2] || (a3 != a2);
      }
    }
  }
  for (int i = 0; i < kPrMaxPerLaunch; ++i)
    if (__any_sync(0xffffffffu, ch[i]) && (threadIdx.x & 31) == 0) changed[i] = 1;
}

__global__ void k_pr_fill_u64(int64_t n, unsigned long long* __restrict__ p) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    p[v] = ~0ull;
}

// Eligible arcs propose themselves to their tree (arc-centric tiles).
template <class OffT>
__global__ void __launch_bounds__(kArcThreads) k_pr_hook(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                                                         int64_t n, int64_t A, const int32_t* __restrict__ tile_row,
                                                         const int32_t* __restrict__ rep, int max_rule,
                                                         unsigned long long* __restrict__ best) {
  __shared__ __align__(16) int32_t s_row[kArcTile];
  for (int64_t a0 = (int64_t)blockIdx.x * kArcTile; a0 < A; a0 += (int64_t)gridDim.x * kArcTile) {
    const int cnt = (int)(A - a0 < kArcTile ? A - a0 : kArcTile);
    const int64_t t = a0 / kArcTile;
    arc_tile_rows(off, n, a0, cnt, s_row, tile_row[t], tile_row[t + 1]);
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      if (i < cnt) {
        const int32_t u = s_row[i];
        const int32_t v = col[a0 + i];
        const int32_t ru = rep[u], rv = rep[v];
        if (ru != rv && (max_rule ? rv > ru : rv < ru))
          atomicMin(&best[ru], ((unsigned long long)(uint32_t)u << 32) | (uint32_t)v);
      }
    }
    __syncthreads();
  }
}

// The same proposals from a list of undirected edges (both orientations):
// the arcs of an insertion batch.
__global__ void k_pr_hook_edges(int64_t k, const int32_t* __restrict__ uv, int64_t n,
                                const int32_t* __restrict__ rep, int max_rule,
                                unsigned long long* __restrict__ best, uint32_t* status) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = uv[2 * j], b = uv[2 * j + 1];
    if (a < 0 || b < 0 || (int64_t)a >= n || (int64_t)b >= n) {
      raise_error(status, DERR_INDEX);
      continue;
    }
    const int32_t ra = rep[a], rb = rep[b];
    if (ra == rb) continue;
    if (max_rule ? rb > ra : rb < ra)
      atomicMin(&best[ra], ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b);
    else
      atomicMin(&best[rb], ((unsigned long long)(uint32_t)b << 32) | (uint32_t)a);
  }
}

// A given starting forest: copied in, parents checked against [0, n).
__global__ void k_pr_load(int64_t n, const int32_t* __restrict__ init, int32_t* __restrict__ P, uint32_t* status) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = init[v];
    if (p < 0 || (int64_t)p >= n) {
      raise_error(status, DERR_INDEX);
      p = (int32_t)v;
    }
    P[v] = p;
  }
}

// Hooking roots start their paths: the bottom vertex u is marked and
// remembers its graft target.
__global__ void k_pr_start(int64_t n, const int32_t* __restrict__ P, const unsigned long long* __restrict__ best,
                           uint8_t* __restrict__ mark, int32_t* __restrict__ graft, unsigned long long* hooks) {
  unsigned long long cnt = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    if (P[r] != (int32_t)r) continue;
    const unsigned long long b = best[r];
    if (b == ~0ull) continue;
    const int32_t u = (int32_t)(b >> 32), v = (int32_t)(b & 0xffffffffull);
    mark[u] = 1;
    graft[u] = v;
    ++cnt;
  }
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(hooks, cnt);
}

// Marks spread one level: x marked => its 2^k-th ancestor marked.
__global__ void k_pr_spread(int64_t n, const int32_t* __restrict__ anc, uint8_t* __restrict__ mark) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    if (mark[x]) mark[anc[x]] = 1;
}

// Q[P[x]] = x for marked non-roots, Q[u] = graft target for path bottoms,
// Q[x] = P[x] for unmarked vertices.  Clears the marks for the next round.
__global__ void k_pr_reverse(int64_t n, const int32_t* __restrict__ P, int32_t* __restrict__ Q,
                             uint8_t* __restrict__ mark, int32_t* __restrict__ graft) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = P[x];
    if (!mark[x]) {
      Q[x] = p;
      continue;
    }
    if (p != (int32_t)x) Q[p] = (int32_t)x;
    const int32_t g = graft[x];
    if (g >= 0) {
      Q[x] = g;
      graft[x] = -1;
    }
    mark[x] = 0;
  }
}

// Minimum vertex of every tree that does not contain the root.
__global__ void k_pr_minv(int64_t n, const int32_t* __restrict__ rep, int32_t root_tree, int32_t* __restrict__ mn) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rep[v];
    if (r != root_tree) atomicMin(&mn[r], (int32_t)v);
  }
}

// Final re-rooting targets: root for its tree, the minimum vertex otherwise.
__global__ void k_pr_targets(int64_t n, const int32_t* __restrict__ P, int32_t root, int32_t root_tree,
                             const int32_t* __restrict__ mn, uint8_t* __restrict__ mark, int32_t* __restrict__ graft) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    if (P[r] != (int32_t)r) continue;
    const int32_t t = (r == root_tree) ? root : mn[r];
    if (t != (int32_t)r) {
      mark[t] = 1;
      graft[t] = t;
    }
  }
}

__global__ void k_pr_fill_i32(int64_t n, int32_t* __restrict__ p, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ---- sparse rounds (small insertion batches) ------------------------------
// The same rounds with work proportional to the batch instead of n: each end
// of an inserted edge finds its tree's root by walking up (at most `limit`
// steps), hooks go to per-root slots, and each hooking tree reverses its own
// path u -> root in place (paths of different trees are disjoint, so the
// result equals the data-parallel reversal).  A walk longer than `limit` sets
// *fallback and the round changes nothing: the caller continues with the
// dense rounds from the same forest and round index.

// Slot e of the batch's ends (uv[e]): its root, and the root's hook slot and
// claim word reset.
__global__ void k_sp_roots(int64_t ends, const int32_t* __restrict__ uv, int64_t n, const int32_t* __restrict__ P,
                           int32_t* __restrict__ rep_e, unsigned long long* __restrict__ best,
                           int32_t* __restrict__ claim, int64_t limit, int32_t* fallback, uint32_t* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ends; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = uv[e];
    if (x < 0 || (int64_t)x >= n) {
      raise_error(status, DERR_INDEX);
      rep_e[e] = -1;
      continue;
    }
    int32_t r = x;
    int64_t steps = 0;
    bool ok = true;
    while (true) {
      const int32_t p = P[r];
      if (p == r) break;
      if (p < 0 || (int64_t)p >= n) {
        raise_error(status, DERR_INDEX);
        ok = false;
        break;
      }
      if (++steps > limit) {
        *fallback = 1;
        ok = false;
        break;
      }
      r = p;
    }
    rep_e[e] = ok ? r : -1;
    if (ok) {
      best[r] = ~0ull;
      claim[r] = 0;
    }
  }
}

// Proposals of the inserted edges (both orientations), as k_pr_hook_edges.
__global__ void k_sp_hook(int64_t k, const int32_t* __restrict__ uv, const int32_t* __restrict__ rep_e, int max_rule,
                          unsigned long long* __restrict__ best, const int32_t* __restrict__ fallback) {
  if (*fallback) return;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = uv[2 * j], b = uv[2 * j + 1];
    const int32_t ra = rep_e[2 * j], rb = rep_e[2 * j + 1];
    if (ra < 0 || rb < 0 || ra == rb) continue;
    if (max_rule ? rb > ra : rb < ra)
      atomicMin(&best[ra], ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b);
    else
      atomicMin(&best[rb], ((unsigned long long)(uint32_t)b << 32) | (uint32_t)a);
  }
}

// The end that is its tree's chosen bottom vertex u (claimed once, ends may
// repeat) reverses the path u -> root and grafts u under v: one thread per
// hooking tree.  The path was walked by k_sp_roots within the step limit.
__global__ void k_sp_reverse(int64_t ends, const int32_t* __restrict__ uv, const int32_t* __restrict__ rep_e,
                             int32_t* __restrict__ P, const unsigned long long* __restrict__ best,
                             int32_t* __restrict__ claim, int64_t limit, const int32_t* __restrict__ fallback,
                             unsigned long long* hooks, uint32_t* status) {
  if (*fallback) return;
  unsigned long long cnt = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ends; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rep_e[e];
    if (r < 0) continue;
    const unsigned long long bk = best[r];
    if (bk == ~0ull) continue;
    const int32_t u = (int32_t)(bk >> 32), v = (int32_t)(bk & 0xffffffffull);
    if (uv[e] != u || atomicExch(&claim[r], 1) != 0) continue;
    int32_t cur = u, np = v;
    for (int64_t steps = 0; steps <= limit; ++steps) {
      const int32_t old = P[cur];
      P[cur] = np;
      if (old == cur) break;
      np = cur;
      cur = old;
    }
    ++cnt;
  }
  (void)status;
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(hooks, cnt);
}

// ---- sparse final re-rooting (the caller declares the input canonical) ----
// Every tree of the input not holding `root` is rooted at its minimum vertex
// and the one holding `root` at root, so only trees the batch merged need
// re-rooting: a merged tree not holding root at the smallest original root
// among its parts, the tree holding root at root.  Ends are the batch's 2k
// ends plus `root` itself (slot 2k).

__device__ __forceinline__ int32_t sp_end(const int32_t* __restrict__ uv, int64_t ends, int32_t root, int64_t e) {
  return e < ends ? uv[e] : root;
}

// Current root of every end (bounded walk); the merged trees' slots reset.
__global__ void k_sp_final_roots(int64_t ends, const int32_t* __restrict__ uv, int32_t root, int64_t n,
                                 const int32_t* __restrict__ P, int32_t* __restrict__ cur_e,
                                 int32_t* __restrict__ tmin, int32_t* __restrict__ claim, int64_t limit,
                                 int32_t* fallback) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= ends; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = sp_end(uv, ends, root, e);
    int32_t r = -1;
    if (x >= 0 && (int64_t)x < n) {
      r = x;
      for (int64_t steps = 0;; ++steps) {
        const int32_t p = P[r];
        if (p == r) break;
        if (steps >= limit || p < 0 || (int64_t)p >= n) {
          *fallback = 1;
          r = -1;
          break;
        }
        r = p;
      }
    }
    cur_e[e] = r;
    if (r >= 0) {
      tmin[r] = INT_MAX;
      claim[r] = 0;
    }
  }
}

// The smallest original root among each merged tree's parts (-1 marks the
// tree holding root: its target is root).
__global__ void k_sp_final_min(int64_t ends, const int32_t* __restrict__ cur_e, const int32_t* __restrict__ orig_e,
                               int32_t* __restrict__ tmin) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= ends; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cur_e[e];
    if (c < 0) continue;
    atomicMin(&tmin[c], e == ends ? -1 : orig_e[e]);
  }
}

// One thread per merged tree re-roots it at its target: the path target ->
// current root is walked once read-only (within the limit, else the dense
// re-rooting takes over and this tree is left alone), then reversed.
__global__ void k_sp_final_reverse(int64_t ends, const int32_t* __restrict__ cur_e, const int32_t* __restrict__ tmin,
                                   int32_t root, int32_t* __restrict__ P, int32_t* __restrict__ claim, int64_t limit,
                                   int32_t* fallback) {
  if (*fallback) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= ends; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cur_e[e];
    if (c < 0 || atomicExch(&claim[c], 1) != 0) continue;
    const int32_t t = tmin[c] < 0 ? root : tmin[c];
    if (t == c) continue;
    int32_t x = t;
    bool ok = false;
    for (int64_t steps = 0; steps <= limit; ++steps) {
      const int32_t p = P[x];
      if (p == x) {
        ok = (x == c);
        break;
      }
      x = p;
    }
    if (!ok) {
      *fallback = 1;
      continue;
    }
    int32_t cur = t, np = t;
    for (int64_t steps = 0; steps <= limit; ++steps) {
      const int32_t old = P[cur];
      P[cur] = np;
      if (old == cur) break;
      np = cur;
      cur = old;
    }
  }
}

struct PrBufs {
  int32_t* anc[kPrMaxLevels];  // anc[0] is P
  int32_t* Q;
  unsigned long long* best;
  uint8_t* mark;
  int32_t* graft;
  int32_t* mn;
  int32_t* tile_row;
  int32_t* flag;
  int levels;
};

// anc[1..K] by pointer jumping until nothing changes; returns K (rep = anc[K]).
// tuning().pr_levels levels are computed per launch (and per host check).
static rst_status pr_history(PrBufs& b, int64_t n, cudaStream_t s, int* K_out) {
  const int g = grid_for(n);
  const int per = tuning().pr_levels;
  int k = 0;
  while (true) {
    if (k + 1 >= b.levels) return RST_ERR_NOT_CONVERGED;
    int j = per;
    if (k + j >= b.levels) j = b.levels - 1 - k;
    RST_CUDA(cudaMemsetAsync(b.flag, 0, kPrMaxPerLaunch * sizeof(int32_t), s));
    if (j == 1) {
      RST_LAUNCH(k_pr_jump, g, kBlock, 0, s)(n, b.anc[k], b.anc[k + 1], b.flag);
    } else {
      RST_LAUNCH(k_pr_jump_multi, g, kBlock, 0, s)(n, b.anc[k], b.anc[k + 1], b.anc[k + 2],
                                                   j >= 3 ? b.anc[k + 3] : nullptr, j, b.flag);
    }
    int32_t changed[kPrMaxPerLaunch] = {0, 0, 0};
    RST_CUDA(cudaMemcpyAsync(host_scratch(16), b.flag, j * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RST_CUDA(cudaStreamSynchronize(s));
    std::memcpy(changed, host_scratch(16), j * sizeof(int32_t));
    int i = 0;
    while (i < j && changed[i]) ++i;
    if (i < j) {  // level k+i+1 equals level k+i: the fixed point
      k += i + 1;
      break;
    }
    k += j;
  }
  *K_out = k;
  return RST_OK;
}

// Spread the marks over levels K-1..0, then reverse into Q and swap P <-> Q.
static rst_status pr_reverse(PrBufs& b, int64_t n, int K, cudaStream_t s) {
  const int g = grid_for(n);
  for (int k = K - 1; k >= 0; --k) RST_LAUNCH(k_pr_spread, g, kBlock, 0, s)(n, b.anc[k], b.mark);
  RST_LAUNCH(k_pr_reverse, g, kBlock, 0, s)(n, b.anc[0], b.Q, b.mark, b.graft);
  std::swap(b.anc[0], b.Q);
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}

// PR-RST rounds over the arcs of a CSR (off/col, A arcs) or, when uv is set,
// over the k undirected edges of uv; from singletons, or from the rooted
// forest `init` when it is set.
template <class OffT>
rst_status prrst_impl(const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root, int32_t* parent,
                      cudaStream_t s, const int32_t* init = nullptr, const int32_t* uv = nullptr, int64_t k = 0,
                      bool canonical = false) {
  int levels = 2;
  while (((int64_t)1 << (levels - 2)) < n + 1 && levels < kPrMaxLevels) ++levels;
  const int64_t tiles = (A + kArcTile - 1) / kArcTile;
  auto al = [](size_t x) { return (x + 255) / 256 * 256 + 256; };
  const size_t ws = al(n * 4) * (levels + 1) + al(n * 8) + al(n) + al(n * 4) * 2 + al((tiles + 2) * 4) + 256 +
                    (uv ? al(2 * (size_t)k * 4) + al(4) + 2 * al((2 * (size_t)k + 1) * 4) + al(4) + al(n * 4) : 0);
  RST_TRY(ensure_workspace(ws));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  PrBufs b{};
  b.levels = levels;
  for (int k = 0; k < levels; ++k) b.anc[k] = ar.take<int32_t>(n);
  b.Q = ar.take<int32_t>(n);
  b.best = ar.take<unsigned long long>(n);
  b.mark = ar.take<uint8_t>(n);
  b.graft = ar.take<int32_t>(n);
  b.mn = ar.take<int32_t>(n);
  b.tile_row = ar.take<int32_t>(tiles + 2);
  b.flag = ar.take<int32_t>(kPrMaxPerLaunch);
  if (!b.flag) return RST_ERR_OOM;
  unsigned long long* hooks = dev_counter(0);
  const int g = grid_for(n);
  uint32_t* status = st.status;
  if (init)
    RST_LAUNCH(k_pr_load, g, kBlock, 0, s)(n, init, b.anc[0], status);
  else
    RST_LAUNCH(k_pr_iota, g, kBlock, 0, s)(n, b.anc[0]);
  RST_CUDA(cudaMemsetAsync(b.mark, 0, n, s));
  RST_LAUNCH(k_pr_fill_i32, g, kBlock, 0, s)(n, b.graft, -1);
  if (!uv && A > 0)
    RST_LAUNCH(k_arc_tile_rows<OffT>, grid_for(tiles + 1), kBlock, 0, s)(off, n, A, tiles, b.tile_row);
  int round = 0;
  bool rounds_done = false;
  const int64_t walk_limit = tuning().insert_walk_limit;
  // canonical input: the original root of every end (and of root), taken
  // before any round changes the forest, for a sparse final re-rooting
  int32_t* orig_e = nullptr;
  int32_t* cur_e = nullptr;
  int32_t* ffb = nullptr;
  int32_t* fclaim = nullptr;  // claim words of the final step (n)
  bool sparse_final = false;
  if (uv && canonical && walk_limit > 0 && k * 64 <= n) {
    orig_e = ar.take<int32_t>(2 * k + 1);
    cur_e = ar.take<int32_t>(2 * k + 1);
    ffb = ar.take<int32_t>(1);
    fclaim = ar.take<int32_t>(n);
    if (ar.used > ar.cap) return RST_ERR_OOM;
    RST_CUDA(cudaMemsetAsync(ffb, 0, sizeof(int32_t), s));
    // the slots it resets (mn, fclaim) are reset again before any use
    RST_LAUNCH(k_sp_final_roots, grid_for(2 * k + 1), kBlock, 0, s)(2 * k, uv, root, n, b.anc[0], orig_e, b.mn,
                                                                   fclaim, walk_limit, ffb);
    sparse_final = true;
  }
  if (uv && k > 0 && walk_limit > 0 && k * 64 <= n) {
    // sparse rounds while every end's walk to its root stays short
    int32_t* rep_e = ar.take<int32_t>(2 * k);
    int32_t* fb = ar.take<int32_t>(1);
    if (ar.used > ar.cap) return RST_ERR_OOM;
    RST_CUDA(cudaMemsetAsync(fb, 0, sizeof(int32_t), s));
    const int ge = grid_for(2 * k);
    for (;; ++round) {
      if (round >= kPrMaxRounds) return RST_ERR_NOT_CONVERGED;
      RST_CUDA(cudaMemsetAsync(hooks, 0, sizeof(unsigned long long), s));
      RST_LAUNCH(k_sp_roots, ge, kBlock, 0, s)(2 * k, uv, n, b.anc[0], rep_e, b.best, b.mn, walk_limit, fb, status);
      RST_LAUNCH(k_sp_hook, grid_for(k), kBlock, 0, s)(k, uv, rep_e, round & 1, b.best, fb);
      RST_LAUNCH(k_sp_reverse, ge, kBlock, 0, s)(2 * k, uv, rep_e, b.anc[0], b.best, b.mn, walk_limit, fb, hooks,
                                                status);
      RST_CUDA(cudaGetLastError());
      unsigned long long hf[2] = {0, 0};
      RST_CUDA(cudaMemcpyAsync(host_scratch(16), hooks, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      RST_CUDA(cudaMemcpyAsync((char*)host_scratch(16) + 8, fb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RST_CUDA(cudaStreamSynchronize(s));
      std::memcpy(hf, host_scratch(16), 12);
      if ((int32_t)hf[1] != 0) break;  // a long walk: the dense rounds take over at this round
      if (hf[0] == 0) {
        rounds_done = true;
        break;
      }
    }
  }
  for (; !rounds_done; ++round) {
    if (round >= kPrMaxRounds) return RST_ERR_NOT_CONVERGED;
    int K = 0;
    RST_TRY(pr_history(b, n, s, &K));
    const int32_t* rep = b.anc[K];
    RST_LAUNCH(k_pr_fill_u64, g, kBlock, 0, s)(n, b.best);
    if (uv) {
      if (k > 0)
        RST_LAUNCH(k_pr_hook_edges, grid_for(k), kBlock, 0, s)(k, uv, n, rep, round & 1, b.best, status);
    } else if (A > 0) {
      RST_LAUNCH(k_pr_hook<OffT>, (unsigned)tiles, kArcThreads, 0, s)(off, col, n, A, b.tile_row, rep, round & 1,
                                                                    b.best);
    }
    RST_CUDA(cudaMemsetAsync(hooks, 0, sizeof(unsigned long long), s));
    RST_LAUNCH(k_pr_start, g, kBlock, 0, s)(n, b.anc[0], b.best, b.mark, b.graft, hooks);
    unsigned long long h = 0;
    RST_TRY(fetch_u64(hooks, 1, &h, s));
    if (h == 0) break;
    RST_TRY(pr_reverse(b, n, K, s));
  }
  if (sparse_final) {
    const int ge = grid_for(2 * k + 1);
    RST_LAUNCH(k_sp_final_roots, ge, kBlock, 0, s)(2 * k, uv, root, n, b.anc[0], cur_e, b.mn, fclaim, walk_limit,
                                                   ffb);
    RST_LAUNCH(k_sp_final_min, ge, kBlock, 0, s)(2 * k, cur_e, orig_e, b.mn);
    RST_LAUNCH(k_sp_final_reverse, ge, kBlock, 0, s)(2 * k, cur_e, b.mn, root, b.anc[0], fclaim, walk_limit, ffb);
    RST_CUDA(cudaGetLastError());
    int32_t f = 0;
    RST_CUDA(cudaMemcpyAsync(host_scratch(4), ffb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RST_CUDA(cudaStreamSynchronize(s));
    std::memcpy(&f, host_scratch(4), sizeof(int32_t));
    if (f == 0) {
      RST_CUDA(cudaMemcpyAsync(parent, b.anc[0], n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      set_stat(STAT_ROUNDS, round + 1);
      return read_device_error(s);
    }
    // a long walk: every tree is re-rooted by the dense step below
  }
  // final re-rooting
  int K = 0;
  RST_TRY(pr_history(b, n, s, &K));
  int32_t root_tree = 0;
  RST_CUDA(cudaMemcpyAsync(host_scratch(4), b.anc[K] + root, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaStreamSynchronize(s));
  std::memcpy(&root_tree, host_scratch(4), sizeof(int32_t));
  RST_LAUNCH(k_pr_fill_i32, g, kBlock, 0, s)(n, b.mn, INT_MAX);
  RST_LAUNCH(k_pr_minv, g, kBlock, 0, s)(n, b.anc[K], root_tree, b.mn);
  RST_LAUNCH(k_pr_targets, g, kBlock, 0, s)(n, b.anc[0], root, root_tree, b.mn, b.mark, b.graft);
  RST_TRY(pr_reverse(b, n, K, s));
  RST_CUDA(cudaMemcpyAsync(parent, b.anc[0], n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  set_stat(STAT_ROUNDS, round + 1);
  return read_device_error(s);
}

}  // namespace

rst_status run_prrst(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m, int32_t root,
                     int32_t* parent, cudaStream_t s) {
  if (offsets_bits == 32) return prrst_impl<int32_t>((const int32_t*)off, cols, n, m, root, parent, s);
  return prrst_impl<int64_t>((const int64_t*)off, cols, n, m, root, parent, s);
}

rst_status run_prrst_insert(int64_t n, int32_t* parent, const int32_t* uv, int64_t k, int32_t root,
                            bool canonical, cudaStream_t s) {
  // the rounds read the starting forest from `parent` and write the result
  // back to it at the end (the copy into the history buffers comes first)
  return prrst_impl<int32_t>(nullptr, nullptr, n, 0, root, parent, s, parent, uv, k, canonical);
}

}  // namespace rst
