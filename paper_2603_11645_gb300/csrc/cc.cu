// Connected components with spanning-forest marking (Section III-B).
//
// Hooking rule (the paper leaves GConn's rule open): Boruvka-style minimum-key
// hooking with edge key (min(u,v), max(u,v)).  Keys are distinct, so the hooks
// of one round form a forest once each mutual pair (two components that chose
// the same edge) keeps its smaller id as root; every successful hook marks
// its edge as a spanning edge.  The marked set is therefore exactly the
// unique minimum spanning forest under those keys (the cut property), the
// same set Kruskal's algorithm yields.  Pointer jumping then flattens each
// hooked tree so that every member points at its root.
//
// GB300 layout choices:
//  * Round 1 works on vertices: with sorted rows the minimum-key edge of a
//    vertex is the arc to its first neighbour, so no atomics are needed; a
//    single kernel resolves mutual pairs, records the tree edges and
//    compresses the hook forest (in-place shortcutting to the root).
//  * Later rounds run on a contracted graph: components get dense ids and the
//    surviving inter-component edges form a shrinking list {cu, cv, p} (p =
//    CSR position of the edge's arc min->max, an order-preserving 32-bit key).
//    Hooking is one packed 64-bit atomicMin per endpoint: high word = key,
//    low word = the other component, so the winner also names its target.
//    All per-component arrays are dense and small, hence L2-resident.
//  * Tree edges are recorded as {p, q, a, b} plus two bits in a bitmap over
//    CSR positions; the Euler stage turns the bitmap into the lexicographically
//    sorted tree-arc order without a sort.
#include <climits>

#include "csr_walk.cuh"
#include "pipeline.cuh"

namespace rst {

constexpr int kMaxRounds = 64;
constexpr int32_t kFinal = -1;

struct CcBuffers {
  int32_t* P;        // n: round-1 hook target, then root
  uint32_t* J;       // n: CSR position of the arc to the first neighbour (kNone: isolated)
  int32_t* CID;      // n: dense component id of round-1 roots
  int32_t* C1;       // n: round-1 component of each vertex (-1: isolated)
  int32_t* Ecu[2];   // list entries (ping-pong)
  int32_t* Ecv[2];
  uint32_t* Ep[2];
  unsigned long long* best;  // n/2+1
  int32_t* P2;       // n/2+1
  int32_t* NID;      // n/2+1
  int32_t* nextpool; // n+1: per-round component maps
  int32_t* minvpool; // n+1: per-round minimum vertex ids (then labels)
  uint4* pairs;      // n
  uint32_t* bits;    // A/32 + 1
  int32_t* roots;    // n/2+1
  int64_t ecap;      // list capacity
};

static CcBuffers cc_layout(Arena& ar, int64_t n, int64_t A) {
  CcBuffers b{};
  int64_t half = n / 2 + 1;
  b.P = ar.take<int32_t>(n + 1);
  b.J = ar.take<uint32_t>(n + 1);
  b.CID = ar.take<int32_t>(n + 1);
  b.C1 = ar.take<int32_t>(n + 1);
  b.ecap = A / 2 + 1;
  for (int k = 0; k < 2; ++k) {
    b.Ecu[k] = ar.take<int32_t>(b.ecap);
    b.Ecv[k] = ar.take<int32_t>(b.ecap);
    b.Ep[k] = ar.take<uint32_t>(b.ecap);
  }
  b.best = ar.take<unsigned long long>(half);
  b.P2 = ar.take<int32_t>(half);
  b.NID = ar.take<int32_t>(half);
  b.nextpool = ar.take<int32_t>(n + 1);
  b.minvpool = ar.take<int32_t>(n + 1);
  b.pairs = ar.take<uint4>(n + 1);
  b.bits = ar.take<uint32_t>(A / 32 + 2);
  b.roots = ar.take<int32_t>(half);
  return b;
}

template <class OffT>
size_t cc_workspace_bytes(int64_t n, int64_t A) {
  Arena a;
  a.counting = true;
  cc_layout(a, n, A);
  return a.used;
}

// counters (64-bit device words)
enum { CNT_PAIRS = 0, CNT_COMPS = 1, CNT_LIST = 2, CNT_ROOTS = 3, CNT_NEXT = 4, CNT_ROOTLABEL = 5 };

// ------------------------------------------------------------------ round 1

// P[u] = first neighbour of u other than u itself (the endpoint of u's
// minimum-key edge: rows are sorted), J[u] = its CSR position; isolated
// vertices point at themselves with J = kNone.
template <class OffT>
__global__ void k_r1_choose(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                            int64_t n, int32_t* __restrict__ P, uint32_t* __restrict__ J,
                            uint32_t* status) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = (int64_t)off[u], hi = (int64_t)off[u + 1];
    while (j < hi && col[j] == (int32_t)u) ++j;
    int32_t v0 = (int32_t)u;
    uint32_t jj = kNone;
    if (j < hi) {
      int32_t c = col[j];
      if (c < 0 || (int64_t)c >= n) {
        raise_error(status, DERR_INDEX);
      } else {
        v0 = c;
        jj = (uint32_t)j;
      }
    }
    P[u] = v0;
    J[u] = jj;
  }
}

// Resolve round 1: u is a root iff it is isolated or the smaller end of a
// mutual pair.  Every other vertex hooked through its edge {u, P[u]}: record
// the tree edge and shortcut u to its root (in place; any value a concurrent
// reader sees is an ancestor, and a 2-cycle is a mutual pair whose smaller id
// is the root).
template <class OffT>
__global__ void k_r1_resolve(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                             int64_t n, int32_t* P, const uint32_t* __restrict__ J,
                             uint4* __restrict__ pairs, uint32_t* __restrict__ bits,
                             unsigned long long* counters, uint32_t* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t u = base + threadIdx.x;
    bool emit = false;
    uint4 rec = make_uint4(0, 0, 0, 0);
    if (u < n) {
      const int32_t v0 = P[u];  // only this thread writes P[u]
      if (v0 != (int32_t)u) {
        const bool mutual = (P[v0] == (int32_t)u);
        const bool is_root = mutual && (int32_t)u < v0;
        if (is_root) {
          P[u] = (int32_t)u;
        } else {
          int64_t q = row_find(off, col, v0, (int32_t)u);
          if (q < 0) {
            raise_error(status, DERR_INDEX);  // the CSR is not symmetric
          } else {
            emit = true;
            rec = make_uint4(J[u], (uint32_t)q, (uint32_t)u, (uint32_t)v0);
            atomicOr(&bits[rec.x >> 5], 1u << (rec.x & 31));
            atomicOr(&bits[rec.y >> 5], 1u << (rec.y & 31));
          }
          // chase to the root
          int32_t x = v0, r = -1;
          for (int64_t it = 0; it <= n; ++it) {
            const int32_t y = P[x];
            if (y == x) { r = x; break; }
            const int32_t z = P[y];
            if (z == x) { r = x < y ? x : y; break; }
            x = y;
          }
          if (r < 0) {
            raise_error(status, DERR_ROUND_LIMIT);
            r = (int32_t)u;
          }
          P[u] = r;
        }
      }
    }
    const unsigned long long slot = block_reserve<kBlock>(&counters[CNT_PAIRS], emit ? 1u : 0u);
    if (emit) pairs[slot] = rec;
  }
}

// Dense ids for round-1 roots that have edges.  The root of a round-1
// component is its minimum vertex (the minimum vertex w hooks to its first
// neighbour x, whose first neighbour is w), so minv starts as the root id.
__global__ void k_r1_number(int64_t n, const int32_t* __restrict__ P,
                            const uint32_t* __restrict__ J, int32_t* __restrict__ CID,
                            int32_t* __restrict__ minv, unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    bool is_root = false;
    if (v < n) is_root = (P[v] == (int32_t)v) && (J[v] != kNone);
    const unsigned long long id = block_reserve<kBlock>(&counters[CNT_COMPS], is_root ? 1u : 0u);
    if (is_root) {
      CID[v] = (int32_t)id;
      minv[id] = (int32_t)v;
    }
  }
}

__global__ void k_r1_label(int64_t n, const int32_t* __restrict__ P, const uint32_t* __restrict__ J,
                           const int32_t* __restrict__ CID, int32_t* __restrict__ C1) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    C1[v] = (J[v] == kNone) ? -1 : CID[P[v]];
  }
}

// The inter-component edges after round 1: every arc u->v with u < v whose
// endpoints lie in different round-1 components, as {C1[u], C1[v], position}.
template <class OffT>
struct BuildListFn {
  const int32_t* __restrict__ col;
  const int32_t* __restrict__ C1;
  int64_t n;
  int32_t* __restrict__ Ecu;
  int32_t* __restrict__ Ecv;
  uint32_t* __restrict__ Ep;
  unsigned long long* counter;
  int64_t cap;
  uint32_t* status;
  // per-thread staging of one tile's kept entries (registers after unrolling)
  int32_t bu[kMpItems], bv[kMpItems];
  uint32_t bp[kMpItems];
  uint32_t mask;
  __device__ __forceinline__ void operator()(int it, bool is_arc, int64_t row, int64_t arc) {
    if (it == 0) mask = 0;
    if (is_arc) {
      const int32_t v = col[arc];
      if (v < 0 || (int64_t)v >= n) {
        raise_error(status, DERR_INDEX);
      } else if (v > (int32_t)row) {
        const int32_t cu = C1[row];
        const int32_t cv = C1[v];
        bu[it] = cu;
        bv[it] = cv;
        bp[it] = (uint32_t)arc;
        if (cu != cv) mask |= 1u << it;
      }
    }
  }
  __device__ __forceinline__ void end_tile() {
    unsigned long long slot = block_reserve<kMpThreads>(counter, (unsigned)__popc(mask));
#pragma unroll
    for (int it = 0; it < kMpItems; ++it) {
      if (mask & (1u << it)) {
        if ((int64_t)slot < cap) {
          Ecu[slot] = bu[it];
          Ecv[slot] = bv[it];
          Ep[slot] = bp[it];
        } else {
          raise_error(status, DERR_CAPACITY);
        }
        ++slot;
      }
    }
  }
};

template <class OffT>
__global__ void __launch_bounds__(kMpThreads) k_build_list(const OffT* __restrict__ off, int64_t n,
                                                           int64_t A, BuildListFn<OffT> f) {
  csr_for_each_arc(off, n, A, f);
}

// ------------------------------------------------------------------ rounds >= 2

__global__ void k_fill_u64(unsigned long long* p, int64_t count, unsigned long long v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_fill_i32(int32_t* p, int64_t count, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Packed minimum-key hook: best[c] = min over incident edges of (key << 32 | other).
__global__ void k_hook(int64_t E, const int32_t* __restrict__ Ecu, const int32_t* __restrict__ Ecv,
                       const uint32_t* __restrict__ Ep, unsigned long long* __restrict__ best) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cu = (uint32_t)Ecu[e], cv = (uint32_t)Ecv[e];
    const unsigned long long key = (unsigned long long)Ep[e] << 32;
    atomicMin(&best[cu], key | cv);
    atomicMin(&best[cv], key | cu);
  }
}

// Arc a->b at CSR position p (row a, a unknown, b = col[p]) -> (a, position of b->a).
// In row b, off[col[k]] is non-decreasing in k, and a is the last column x with off[x] <= p.
template <class OffT>
__device__ __forceinline__ bool twin_of_position(const OffT* __restrict__ off,
                                                 const int32_t* __restrict__ col, int32_t b,
                                                 uint64_t p, int32_t* a_out, int64_t* q_out) {
  const int64_t lo = (int64_t)off[b], hi0 = (int64_t)off[b + 1];
  int64_t L = lo, H = hi0;
  while (L < H) {
    const int64_t mid = (L + H) >> 1;
    if ((uint64_t)off[col[mid]] <= p)
      L = mid + 1;
    else
      H = mid;
  }
  const int64_t k = L - 1;
  if (k < lo) return false;
  const int32_t x = col[k];
  if (!((uint64_t)off[x] <= p && p < (uint64_t)off[x + 1])) return false;
  *a_out = x;
  *q_out = k;
  return true;
}

// Resolve one round: a component with no incident edge is final; otherwise it
// hooks onto the component its minimum-key edge reaches, except the smaller id
// of a mutual pair, which stays a root.  Each hook records its tree edge.
template <class OffT>
__global__ void k_resolve(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t C,
                          const unsigned long long* __restrict__ best, int32_t* __restrict__ P2,
                          uint4* __restrict__ pairs, uint32_t* __restrict__ bits,
                          unsigned long long* counters, uint32_t* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < C; base += stride) {
    const int64_t c = base + threadIdx.x;
    bool emit = false;
    uint4 rec = make_uint4(0, 0, 0, 0);
    if (c < C) {
      const unsigned long long b = best[c];
      if (b == ~0ull) {
        P2[c] = (int32_t)c;
      } else {
        const int32_t c2 = (int32_t)(uint32_t)(b & 0xffffffffull);
        const uint32_t p = (uint32_t)(b >> 32);
        const bool mutual = (uint32_t)(best[c2] >> 32) == p;
        if (mutual && (int32_t)c < c2) {
          P2[c] = (int32_t)c;
        } else {
          P2[c] = c2;
          const int32_t bb = col[p];
          int32_t a = 0;
          int64_t q = 0;
          if (twin_of_position(off, col, bb, (uint64_t)p, &a, &q)) {
            emit = true;
            rec = make_uint4(p, (uint32_t)q, (uint32_t)a, (uint32_t)bb);
            atomicOr(&bits[p >> 5], 1u << (p & 31));
            atomicOr(&bits[rec.y >> 5], 1u << (rec.y & 31));
          } else {
            raise_error(status, DERR_INDEX);
          }
        }
      }
    }
    const unsigned long long slot = block_reserve<kBlock>(&counters[CNT_PAIRS], emit ? 1u : 0u);
    if (emit) pairs[slot] = rec;
  }
}

// Pointer jumping over the component forest: shortcut every component to its root.
__global__ void k_compress(int64_t C, int32_t* P2, uint32_t* status) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = P2[c];
    int64_t it = 0;
    while (true) {
      const int32_t y = P2[x];
      if (y == x) break;
      x = y;
      if (++it > C) {
        raise_error(status, DERR_ROUND_LIMIT);
        break;
      }
    }
    P2[c] = x;
  }
}

// New dense ids for the roots that still have edges; components without edges
// are final and their minimum vertex joins the list of component roots.
__global__ void k_renumber(int64_t C, const int32_t* __restrict__ P2,
                           const unsigned long long* __restrict__ best,
                           const int32_t* __restrict__ minv, int32_t* __restrict__ NID,
                           int32_t* __restrict__ roots, unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < C; base += stride) {
    const int64_t c = base + threadIdx.x;
    bool live_root = false, fin = false;
    if (c < C) {
      fin = best[c] == ~0ull;
      live_root = !fin && P2[c] == (int32_t)c;
    }
    const unsigned long long id = block_reserve<kBlock>(&counters[CNT_NEXT], live_root ? 1u : 0u);
    const unsigned long long rid = block_reserve<kBlock>(&counters[CNT_ROOTS], fin ? 1u : 0u);
    if (c < C) NID[c] = live_root ? (int32_t)id : -1;
    if (fin) roots[rid] = minv[c];
  }
}

__global__ void k_map(int64_t C, const int32_t* __restrict__ P2,
                      const unsigned long long* __restrict__ best,
                      const int32_t* __restrict__ NID, const int32_t* __restrict__ minv,
                      int32_t* __restrict__ next, int32_t* __restrict__ minv_next) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (best[c] == ~0ull) {
      next[c] = kFinal;
    } else {
      const int32_t nc = NID[P2[c]];
      next[c] = nc;
      atomicMin(&minv_next[nc], minv[c]);
    }
  }
}

// Relabel the edge list into the next round's ids, dropping edges that now
// join a component to itself.
__global__ void k_relabel(int64_t E, const int32_t* __restrict__ Ecu, const int32_t* __restrict__ Ecv,
                          const uint32_t* __restrict__ Ep, const int32_t* __restrict__ next,
                          int32_t* __restrict__ Ocu, int32_t* __restrict__ Ocv,
                          uint32_t* __restrict__ Op, unsigned long long* counter) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < E; base += stride) {
    const int64_t e = base + threadIdx.x;
    bool keep = false;
    int32_t nu = 0, nv = 0;
    uint32_t p = 0;
    if (e < E) {
      nu = next[Ecu[e]];
      nv = next[Ecv[e]];
      p = Ep[e];
      keep = nu != nv;
    }
    const unsigned long long slot = block_reserve<kBlock>(counter, keep ? 1u : 0u);
    if (keep) {
      Ocu[slot] = nu;
      Ocv[slot] = nv;
      Op[slot] = p;
    }
  }
}

// All components of the last round are final.
__global__ void k_all_final(int64_t C, const int32_t* __restrict__ minv, int32_t* __restrict__ next,
                            int32_t* __restrict__ roots, unsigned long long* counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < C; base += stride) {
    const int64_t c = base + threadIdx.x;
    const bool ok = c < C;
    const unsigned long long rid = block_reserve<kBlock>(&counters[CNT_ROOTS], ok ? 1u : 0u);
    if (ok) {
      roots[rid] = minv[c];
      next[c] = kFinal;
    }
  }
}

// Labels, backwards over rounds: lab_r[c] = minv_r[c] if final, else lab_{r+1}[next_r[c]].
__global__ void k_label_back(int64_t C, const int32_t* __restrict__ next, int32_t* lab_r,
                             const int32_t* __restrict__ lab_next) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t nc = next[c];
    if (nc != kFinal) lab_r[c] = lab_next[nc];
  }
}

__global__ void k_label_vertices(int64_t n, const int32_t* __restrict__ C1,
                                 const int32_t* __restrict__ lab1, int32_t* __restrict__ labels) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = C1[v];
    labels[v] = c < 0 ? (int32_t)v : lab1[c];
  }
}

struct RoundTable {
  int64_t base[kMaxRounds];
  int nrounds;
};

// Canonical label of one vertex by following its component through the rounds.
__global__ void k_root_label(int32_t v, const int32_t* __restrict__ C1,
                             const int32_t* __restrict__ nextpool,
                             const int32_t* __restrict__ minvpool, RoundTable rt,
                             unsigned long long* counters) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int32_t c = C1[v];
  int32_t lab = v;
  if (c >= 0) {
    for (int r = 0; r < rt.nrounds; ++r) {
      const int32_t nc = nextpool[rt.base[r] + c];
      if (nc == kFinal) {
        lab = minvpool[rt.base[r] + c];
        break;
      }
      c = nc;
    }
  }
  counters[CNT_ROOTLABEL] = (unsigned long long)(uint32_t)lab;
}

// ------------------------------------------------------------------ driver

template <class OffT>
rst_status cc_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A,
                  int32_t root, int32_t* labels_out, CcOut* out, cudaStream_t s) {
  CcBuffers b = cc_layout(ar, n, A);
  if (!b.P || !b.roots) return RST_ERR_OOM;
  uint32_t* status = state().status;
  unsigned long long* cnt = dev_counter(0);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  RST_CUDA(cudaMemsetAsync(b.bits, 0, (A / 32 + 2) * sizeof(uint32_t), s));

  const int gN = grid_for(n);
  prof_mark(s, "cc_setup");
  RST_LAUNCH(k_r1_choose<OffT>, gN, kBlock, 0, s)(off, col, n, b.P, b.J, status);
  prof_mark(s, "k_r1_choose");
  RST_LAUNCH(k_r1_resolve<OffT>, gN, kBlock, 0, s)(off, col, n, b.P, b.J, b.pairs, b.bits, cnt, status);
  prof_mark(s, "k_r1_resolve");
  RST_LAUNCH(k_r1_number, gN, kBlock, 0, s)(n, b.P, b.J, b.CID, b.minvpool, cnt);
  prof_mark(s, "k_r1_number");
  RST_LAUNCH(k_r1_label, gN, kBlock, 0, s)(n, b.P, b.J, b.CID, b.C1);
  prof_mark(s, "k_r1_label");
  {
    BuildListFn<OffT> f{col, b.C1, n, b.Ecu[0], b.Ecv[0], b.Ep[0], &cnt[CNT_LIST], b.ecap, status};
    const int64_t tiles = (n + A + kMpTile - 1) / kMpTile;
    const int g = (int)(tiles < (int64_t)device_info().sms * 8 ? (tiles > 0 ? tiles : 1)
                                                                : (int64_t)device_info().sms * 8);
    RST_LAUNCH(k_build_list<OffT>, g, kMpThreads, 0, s)(off, n, A, f);
  }
  prof_mark(s, "k_build_list");
  RST_CUDA(cudaGetLastError());
  unsigned long long h[8];
  RST_TRY(fetch_u64(cnt, 8, h, s));
  prof_mark(s, "cc_sync");
  int64_t C = (int64_t)h[CNT_COMPS];
  int64_t E = (int64_t)h[CNT_LIST];
  set_stat(STAT_C1, C);
  set_stat(STAT_E2, E);
  if (E > b.ecap) return RST_ERR_DEVICE;

  RoundTable rt{};
  int64_t pool_at = 0;  // start of the current round's slice in next/minv pools
  int cur = 0;
  int rounds = 1;
  while (C > 0) {
    if (rt.nrounds >= kMaxRounds) return RST_ERR_NOT_CONVERGED;
    int32_t* minv = b.minvpool + pool_at;
    int32_t* next = b.nextpool + pool_at;
    rt.base[rt.nrounds++] = pool_at;
    const int gC = grid_for(C);
    if (E == 0) {
      RST_LAUNCH(k_all_final, gC, kBlock, 0, s)(C, minv, next, b.roots, cnt);
      RST_CUDA(cudaGetLastError());
      pool_at += C;
      break;
    }
    ++rounds;
    const int gE = grid_for(E);
    RST_LAUNCH(k_fill_u64, gC, kBlock, 0, s)(b.best, C, ~0ull);
    RST_LAUNCH(k_hook, gE, kBlock, 0, s)(E, b.Ecu[cur], b.Ecv[cur], b.Ep[cur], b.best);
    RST_LAUNCH(k_resolve<OffT>, gC, kBlock, 0, s)(off, col, C, b.best, b.P2, b.pairs, b.bits, cnt, status);
    RST_LAUNCH(k_compress, gC, kBlock, 0, s)(C, b.P2, status);
    RST_CUDA(cudaMemsetAsync(&cnt[CNT_NEXT], 0, sizeof(unsigned long long), s));
    RST_LAUNCH(k_renumber, gC, kBlock, 0, s)(C, b.P2, b.best, minv, b.NID, b.roots, cnt);
    RST_CUDA(cudaGetLastError());
    RST_TRY(fetch_u64(cnt, 8, h, s));
    const int64_t Cn = (int64_t)h[CNT_NEXT];
    int32_t* minv_next = b.minvpool + pool_at + C;
    if (pool_at + C + Cn > n + 1) return RST_ERR_DEVICE;
    RST_LAUNCH(k_fill_i32, grid_for(Cn), kBlock, 0, s)(minv_next, Cn, INT_MAX);
    RST_LAUNCH(k_map, gC, kBlock, 0, s)(C, b.P2, b.best, b.NID, minv, next, minv_next);
    RST_CUDA(cudaMemsetAsync(&cnt[CNT_LIST], 0, sizeof(unsigned long long), s));
    RST_LAUNCH(k_relabel, gE, kBlock, 0, s)(E, b.Ecu[cur], b.Ecv[cur], b.Ep[cur], next, b.Ecu[cur ^ 1],
                                    b.Ecv[cur ^ 1], b.Ep[cur ^ 1], &cnt[CNT_LIST]);
    RST_CUDA(cudaGetLastError());
    RST_TRY(fetch_u64(cnt, 8, h, s));
    E = (int64_t)h[CNT_LIST];
    pool_at += C;
    C = Cn;
    cur ^= 1;
  }

  prof_mark(s, "cc_rounds");
  // labels
  if (labels_out) {
    for (int r = rt.nrounds - 2; r >= 0; --r) {
      const int64_t Cr = rt.base[r + 1] - rt.base[r];
      RST_LAUNCH(k_label_back, grid_for(Cr), kBlock, 0, s)(Cr, b.nextpool + rt.base[r],
                                                   b.minvpool + rt.base[r],
                                                   b.minvpool + rt.base[r + 1]);
    }
    RST_LAUNCH(k_label_vertices, gN, kBlock, 0, s)(n, b.C1, b.minvpool, labels_out);
    RST_CUDA(cudaGetLastError());
  }
  out->root_label = -1;
  if (root >= 0) {
    if (labels_out) {
      // the backward pass overwrote minv with labels; read the root's label
      RST_CUDA(cudaMemcpyAsync(&cnt[CNT_ROOTLABEL], labels_out + root, sizeof(int32_t),
                               cudaMemcpyDeviceToDevice, s));
      RST_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(&cnt[CNT_ROOTLABEL]) + 4, 0, 4, s));
    } else {
      RST_LAUNCH(k_root_label, 1, 32, 0, s)(root, b.C1, b.nextpool, b.minvpool, rt, cnt);
      RST_CUDA(cudaGetLastError());
    }
  }
  RST_TRY(fetch_u64(cnt, 8, h, s));
  prof_mark(s, "cc_finish");
  out->T = (int64_t)h[CNT_PAIRS];
  out->pairs = b.pairs;
  out->bits = b.bits;
  out->nroots = (int64_t)h[CNT_ROOTS];
  out->roots = b.roots;
  out->rounds = rounds;
  set_stat(STAT_ROUNDS, rounds);
  set_stat(STAT_T, out->T);
  set_stat(STAT_NROOTS, out->nroots);
  if (root >= 0) out->root_label = (int32_t)(uint32_t)h[CNT_ROOTLABEL];
  return RST_OK;
}

template rst_status cc_run<int32_t>(Arena&, const int32_t*, const int32_t*, int64_t, int64_t,
                                    int32_t, int32_t*, CcOut*, cudaStream_t);
template rst_status cc_run<int64_t>(Arena&, const int64_t*, const int32_t*, int64_t, int64_t,
                                    int32_t, int32_t*, CcOut*, cudaStream_t);
template size_t cc_workspace_bytes<int32_t>(int64_t, int64_t);
template size_t cc_workspace_bytes<int64_t>(int64_t, int64_t);

}  // namespace rst
