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

// Round control in device memory, so that the contraction rounds run without
// host involvement (and can be captured in a CUDA graph).  Round r reads
// st[r] and produces st[r+1].
struct RoundState {
  unsigned long long C;        // components entering the round
  unsigned long long E;        // list entries entering the round (previous round's ids)
  unsigned long long pool_at;  // this round's slice of the next/minv pools
  int rc;                      // the requested root's component (-1: none)
  int bs;                      // stride between this round's hook slots (1 or kSpread)
};
struct CcCtl {
  RoundState st[kMaxRounds + 1];
  // the tail (below): 0 not entered, 1 requested at round tail_round,
  // 2 finished in one block, 3 handed back to the regular rounds
  int tail;
  int tail_round;
  int cur;             // current round
  int root_label;      // canonical label of the requested root (-1 until known)
  unsigned int done;   // blocks of the round's last kernel that have finished
  int tail_rounds;              // rounds the tail ran
  unsigned int tail_hooks;      // tree edges the tail recorded (positions in tp)
  unsigned int tail_overflow;   // the deduplicated pairs did not fit
  int tail_first_back;          // round of the first hand-back (0: none)
  int tail_backs;               // hand-backs
  // the list build (below): the root vertex of a giant round-1 component
  // (-1: none) and the number of vertices with edges outside it
  int giant;
  unsigned int ng;
};

// The tail: once at most kTailC components with edges remain, the list
// (mostly parallel edges between few components by then) is deduplicated to
// one entry per component pair, keeping the smallest key (the minimum-key
// choice of every component depends only on each pair's smallest key), and
// one block finishes all remaining rounds in shared memory.  A tail that does
// not fit (more than kTailPairs distinct pairs) hands back to the regular
// rounds, which continue from the same round and request the tail again one
// round later.  The pair graph of contracted grids and meshes is planar, so
// kTailPairs = 3 kTailC always holds them; contracted random graphs are
// dense and may need one or two more rounds first.
constexpr int kTailC = 3072;
constexpr int kTailPairs = 3 * kTailC;  // a planar pair graph on C vertices has < 3C edges
constexpr int kTailSlots = 16384;  // hash table of component pairs (power of two)
constexpr int kTailProbe = 64;
constexpr int kTailThreads = 1024;
constexpr int kTailBits = 14;     // log2 kTailSlots
constexpr int kTailMaxRounds = 64;
constexpr size_t kTailSmem = (size_t)kTailPairs * 12 + (size_t)kTailC * 32;
static_assert(kTailSlots % kTailThreads == 0, "the table scan takes whole blocks of slots");

// Row record of a vertex, one aligned 32-byte sector: where its row starts,
// its degree and the first kRecCols entries.  Round 1 reads the chosen
// neighbour's record once instead of its pointer, its row bounds and its row.
constexpr int kRecCols = 6;
struct __align__(32) RowRec {
  uint32_t start;
  uint32_t deg;
  int32_t c[kRecCols];
};

struct CcBuffers {
  RowRec* rec;       // per-vertex row records (may be null)
  int32_t* P;        // n: round-1 hook target, then root
  uint32_t* J;       // n: CSR position of the arc to the first neighbour (kNone: isolated)
  uint32_t* rbits;   // n/32 + 2 words: round-1 roots that have edges
  uint2* rrank;      // n/32 + 2: {rbits word, popcount before it} (dense root ids)
  unsigned long long* rtmp;  // scan scratch
  int32_t* C1;       // n: round-1 component of each vertex (-1: isolated)
  int32_t* Ecu[2];   // list entries (ping-pong)
  int32_t* Ecv[2];
  uint32_t* Ep[2];
  unsigned long long* best[2];  // n/2+1 each: round parity
  int32_t* P2;       // n/2+1
  int32_t* NID;      // n/2+1
  int32_t* nextpool; // n+1: per-round component maps
  int32_t* minvpool; // n+1: per-round minimum vertex ids (then labels)
  uint4* pairs;      // n
  uint32_t* bits;    // A/32 + 1
  int32_t* roots;    // n/2+1
  struct CcCtl* ctl; // device-resident round control
  int32_t* tile_row; // row of the first arc of every arc tile
  unsigned long long* tkey;  // kTailSlots: component pair (lo << 32 | hi), ~0 = empty
  uint32_t* tval;            // kTailSlots: smallest key of the pair
  uint32_t* tp;              // kTailC: keys (CSR positions) of the tail's tree edges
  int64_t ecap;      // list capacity
  int64_t bcap;      // slots in each best[] buffer
};

static CcBuffers cc_layout(Arena& ar, int64_t n, int64_t A) {
  CcBuffers b{};
  int64_t half = n / 2 + 1;
  // row records only where the workspace may grow (not in the fixed-scratch
  // variant, whose size limits were set without them)
  b.rec = state_overridden() ? nullptr : ar.take<RowRec>(n + 1);
  b.P = ar.take<int32_t>(n + 1);
  b.J = ar.take<uint32_t>(n + 1);
  b.rbits = ar.take<uint32_t>(n / 32 + 2);
  b.rrank = ar.take<uint2>(n / 32 + 2);
  b.rtmp = ar.take<unsigned long long>(scan_tmp_words(n / 32 + 1));
  b.C1 = ar.take<int32_t>(n + 1);
  b.ecap = A / 2 + 1;
  for (int k = 0; k < 2; ++k) {
    b.Ecu[k] = ar.take<int32_t>(b.ecap);
    b.Ecv[k] = ar.take<int32_t>(b.ecap);
    b.Ep[k] = ar.take<uint32_t>(b.ecap);
  }
  b.bcap = half;
  b.best[0] = ar.take<unsigned long long>(half);
  b.best[1] = ar.take<unsigned long long>(half);
  b.P2 = ar.take<int32_t>(half);
  b.NID = ar.take<int32_t>(half);
  b.nextpool = ar.take<int32_t>(n + 1);
  b.minvpool = ar.take<int32_t>(n + 1);
  b.pairs = ar.take<uint4>(n + 1);
  b.bits = ar.take<uint32_t>(A / 32 + 2);
  b.roots = ar.take<int32_t>(half);
  b.ctl = ar.take<CcCtl>(1);
  b.tile_row = ar.take<int32_t>(A / kArcTile + 2);
  b.tkey = ar.take<unsigned long long>(kTailSlots);
  b.tval = ar.take<uint32_t>(kTailSlots);
  b.tp = ar.take<uint32_t>(kTailC);
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
// vertices point at themselves with J = kNone.  With rs set it also builds
// the row-start bitmap the Euler stage reads (row_start_bit).
template <class OffT>
__global__ void k_r1_choose(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                            int64_t n, int32_t* __restrict__ P, uint32_t* __restrict__ J,
                            RowRec* __restrict__ rec, uint32_t* __restrict__ rs, uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base <= n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = base + threadIdx.x;
    if (rs) row_start_bit(rs, off, n, u, u <= n ? (uint64_t)off[u] : 0, u < n ? (uint64_t)off[u + 1] : 0);
    if (u >= n) continue;
    int64_t j = (int64_t)off[u], hi = (int64_t)off[u + 1];
    if (rec) {
      RowRec r;
      r.start = (uint32_t)j;
      r.deg = (uint32_t)(hi - j);
#pragma unroll
      for (int i = 0; i < kRecCols; ++i) r.c[i] = j + i < hi ? col[j + i] : -1;
      rec[u] = r;
    }
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
// Vertices per thread and step, and the blocks per SM their registers allow:
// two on meshes; three where rows are long (the twin searches of power-law
// graphs gain from the third chain in flight, meshes lose a little).
constexpr int kR1Per = 2, kR1BlocksPerSm = 5;
constexpr int kR1PerLong = 3, kR1BlocksPerSmLong = 4;
constexpr int64_t kR1LongRowDegree = 8;  // arcs per vertex above which rows count as long
template <class OffT, int kPer, int kBps>
__global__ void __launch_bounds__(kBlock, kBps) k_r1_resolve(const OffT* __restrict__ off, const int32_t* __restrict__ col,
                             int64_t n, int32_t* P, const uint32_t* __restrict__ J,
                             const RowRec* __restrict__ rows, uint4* __restrict__ pairs,
                             uint32_t* __restrict__ bits, uint32_t* __restrict__ rbits,
                             unsigned long long* counters, uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  const uint64_t once = l2_evict_first();  // J and the records stream; L2 keeps P and the row records
  const int64_t tile = (int64_t)blockDim.x * kPer;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
    // Every load of a step is issued for both vertices before either is used:
    // own pointers, then the chosen neighbours' records, then the chases in
    // lockstep.  Positions fit 32 bits (fewer than 2^32 arcs).
    int32_t v0[kPer], y[kPer];
    uint32_t act = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int64_t u = base + (int64_t)j * blockDim.x + threadIdx.x;
      v0[j] = u < n ? P[u] : (int32_t)u;  // only this thread writes P[u]
      if (u < n && v0[j] != (int32_t)u) act |= 1u << j;
    }
    // v0's first choice y0 (its first non-self entry) and u's position q in
    // v0's row: from v0's record when it holds the whole row, else from P and
    // a binary search of the row
    uint32_t q[kPer];
    uint32_t haveq = 0;
    if (rows) {
      RowRec R[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j)
        if ((act >> j) & 1u) R[j] = rows[v0[j]];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        y[j] = -1;
        q[j] = kNone;
        if (!((act >> j) & 1u)) continue;
        const int32_t u = (int32_t)(base + (int64_t)j * blockDim.x + threadIdx.x);
#pragma unroll
        for (int i = kRecCols - 1; i >= 0; --i)
          if (i < (int)R[j].deg && R[j].c[i] != v0[j]) y[j] = R[j].c[i];
#pragma unroll
        for (int i = kRecCols - 1; i >= 0; --i)
          if (i < (int)R[j].deg && R[j].c[i] == u) q[j] = R[j].start + (uint32_t)i;
        if (R[j].deg <= (uint32_t)kRecCols) haveq |= 1u << j;
      }
#pragma unroll
      for (int j = 0; j < kPer; ++j)  // long row of self-loops, or a bad id
        if (((act >> j) & 1u) && (y[j] < 0 || (int64_t)y[j] >= n)) y[j] = P[v0[j]];
    } else {
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        y[j] = -1;
        q[j] = kNone;
        if ((act >> j) & 1u) y[j] = P[v0[j]];
      }
    }
    uint32_t emit = 0, chase = 0;
    int32_t x[kPer], root[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      x[j] = 0;
      root[j] = -1;
      if (!((act >> j) & 1u)) continue;
      const int64_t u = base + (int64_t)j * blockDim.x + threadIdx.x;
      const bool mutual = (y[j] == (int32_t)u);
      if (mutual && (int32_t)u < v0[j]) {
        root[j] = (int32_t)u;  // the smaller end of a mutual pair: a root with edges
        if (rbits) atomicOr(&rbits[u >> 5], 1u << (u & 31));
        continue;
      }
      if (!((haveq >> j) & 1u)) {
        const int64_t lo = (int64_t)off[v0[j]], end = (int64_t)off[v0[j] + 1];
        int64_t L = lo, H = end;
        while (L < H) {
          const int64_t mid = (L + H) >> 1;
          if (col[mid] < (int32_t)u)
            L = mid + 1;
          else
            H = mid;
        }
        q[j] = (L < end && col[L] == (int32_t)u) ? (uint32_t)L : kNone;
      }
      if (q[j] == kNone)
        raise_error(status, DERR_INDEX);  // the CSR is not symmetric
      else
        emit |= 1u << j;
      // chase to the root: x -> y = P[x] -> z = P[y]; the first y is y0
      if (mutual) {
        root[j] = v0[j];  // the pair's smaller end (u > v0 here)
      } else {
        x[j] = v0[j];
        chase |= 1u << j;
      }
    }
    for (int64_t it = 0; chase && it <= n; ++it) {
      int32_t z[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        z[j] = 0;
        if ((chase >> j) & 1u) {
          if (y[j] == x[j]) {
            root[j] = x[j];
            chase &= ~(1u << j);
          } else {
            z[j] = P[y[j]];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        if (!((chase >> j) & 1u)) continue;
        if (z[j] == x[j]) {
          root[j] = x[j] < y[j] ? x[j] : y[j];
          chase &= ~(1u << j);
        } else {
          x[j] = y[j];
          y[j] = z[j];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (!((act >> j) & 1u)) continue;
      const int64_t u = base + (int64_t)j * blockDim.x + threadIdx.x;
      if (root[j] < 0) {
        raise_error(status, DERR_ROUND_LIMIT);
        root[j] = (int32_t)u;
        if (rbits) atomicOr(&rbits[u >> 5], 1u << (u & 31));
      }
      P[u] = root[j];
    }
    unsigned wtot = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) wtot += __popc(__ballot_sync(0xffffffffu, (emit >> j) & 1u));
    const unsigned long long mine = block_reserve<kBlock>(&counters[CNT_PAIRS], lane == 0 ? wtot : 0u);
    unsigned long long run = __shfl_sync(0xffffffffu, mine, 0);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const unsigned bal = __ballot_sync(0xffffffffu, (emit >> j) & 1u);
      if ((emit >> j) & 1u) {
        const int64_t u = base + (int64_t)j * blockDim.x + threadIdx.x;
        const uint4 rec = make_uint4(ld_stream(&J[u], once), q[j], (uint32_t)u, (uint32_t)v0[j]);
        atomicOr(&bits[rec.x >> 5], 1u << (rec.x & 31));
        atomicOr(&bits[rec.y >> 5], 1u << (rec.y & 31));
        st_stream(&pairs[run + __popc(bal & lt)], rec, once);
      }
      run += __popc(bal);
    }
  }
}

// A giant round-1 component (power-law graphs: a hub's neighbourhood merges
// in round 1) makes the list build a filter: almost every arc joins two
// vertices of the giant.  A fixed, evenly spaced sample of kGiantSamples
// vertices decides (one block of k_round_init): the roots of kGiantCands
// spread samples are candidates, and the one most samples share is the giant
// when it holds at least `pct` percent of the samples with edges (pct 0: the
// most shared one always).  The choice changes no result, only which rows the
// list build reads.
constexpr int kGiantSamples = 2048;
constexpr int kGiantCands = 32;
constexpr int kGiantMinSamples = 64;  // fewer samples with edges: no giant
// Run by every thread of one kBlock-thread block.
__device__ __forceinline__ void giant_sample(int64_t n, const int32_t* __restrict__ P,
                                             const uint32_t* __restrict__ J, int pct, CcCtl* ctl) {
  constexpr int kPer = kGiantSamples / kBlock;
  static_assert(kPer * kBlock == kGiantSamples && kGiantSamples % kGiantCands == 0, "sample split");
  constexpr int kStep = kGiantSamples / kGiantCands;  // candidate c is sample c * kStep
  __shared__ int32_t s_cand[kGiantCands];
  __shared__ unsigned s_cnt[kGiantCands];
  __shared__ unsigned s_have;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_have = 0;
  if (threadIdx.x < kGiantCands) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  // the samples' roots (-1: isolated), all loads issued together
  int32_t r[kPer];
  uint32_t jv[kPer];
  const bool on = n > 0 && pct <= 100;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = k * kBlock + threadIdx.x;
    const int64_t v = ((2 * (int64_t)i + 1) * n) / (2 * kGiantSamples);
    jv[k] = on ? J[v] : kNone;
    r[k] = on ? P[v] : -1;
  }
  unsigned have = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (jv[k] == kNone) r[k] = -1;
    have += __popc(__ballot_sync(0xffffffffu, r[k] >= 0));
    const int i = k * kBlock + threadIdx.x;
    if (i % kStep == 0) s_cand[i / kStep] = r[k];
  }
  if (lane == 0) atomicAdd(&s_have, have);
  __syncthreads();
  // each sample counts under the first candidate slot holding its root (one
  // shared atomic per distinct slot and warp)
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    int slot = -1;
    if (r[k] >= 0)
      for (int c = 0; c < kGiantCands; ++c)
        if (s_cand[c] == r[k]) {
          slot = c;
          break;
        }
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    if (slot >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[slot], (unsigned)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int c = 1; c < kGiantCands; ++c)
      if (s_cnt[c] > s_cnt[best]) best = c;
    const bool giant = s_have >= (unsigned)kGiantMinSamples && s_cand[best] >= 0 &&
                       100ull * s_cnt[best] >= (unsigned long long)pct * s_have;
    ctl->giant = giant ? s_cand[best] : -1;
    ctl->ng = 0;
  }
}

// Round-1 labels: the dense id of a root with edges is its rank among those
// roots (a popcount prefix over their bitmap, so ids follow vertex order), and
// every non-isolated vertex takes the id of its root.  The root of a round-1
// component is its minimum vertex (the minimum vertex w hooks to its first
// neighbour x, whose first neighbour is w), so minv starts as the root id.
__global__ void k_r1_label(int64_t n, const int32_t* __restrict__ P, const uint32_t* __restrict__ J,
                           const uint2* __restrict__ rrank, int32_t* __restrict__ C1,
                           int32_t* __restrict__ minv, unsigned long long* counters) {
  pdl_wait();  // launched as a programmatic dependent
  if (blockIdx.x == 0 && threadIdx.x == 0) counters[CNT_COMPS] = rrank[n / 32 + 1].y;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = -1;
    if (J[v] != kNone) {
      const int32_t r = P[v];
      c = (int32_t)bit_rank2(rrank, (uint64_t)r);
      if (r == (int32_t)v) minv[c] = (int32_t)v;
    }
    C1[v] = c;
  }
}

// The list is built from the giant's complement when there is a giant.
__device__ __forceinline__ bool sparse_list(const CcCtl* ctl) { return ctl->giant >= 0; }

// The inter-component edges after round 1: every arc u->v with u < v whose
// endpoints lie in different round-1 components, as {C1[u], C1[v], position}.
// The scan also performs the first contraction round's packed atomicMin hook,
// so that round does not read the list again.
// Arc-centric tiles: coalesced column loads, rows from a shared-memory scan,
// independent label gathers, one slot reservation per tile.
template <class OffT>
__global__ void __launch_bounds__(kArcThreads, 6) k_build_list(const OffT* __restrict__ off,
                                                            const int32_t* __restrict__ col,
                                                            int64_t n, int64_t A,
                                                            const int32_t* __restrict__ C1,
                                                            int32_t* __restrict__ Ecu,
                                                            int32_t* __restrict__ Ecv,
                                                            uint32_t* __restrict__ Ep,
                                                            unsigned long long* counter, int64_t cap,
                                                            const int32_t* __restrict__ tile_row,
                                                            unsigned long long* __restrict__ best,
                                                            const CcCtl* ctl, uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  if (sparse_list(ctl)) return;  // k_build_list_sparse builds the list
  __shared__ __align__(16) int32_t s_row[kArcTile];
  const uint64_t once = l2_evict_first();  // the columns stream past; L2 keeps C1 and the hook slots
  for (int64_t a0 = (int64_t)blockIdx.x * kArcTile; a0 < A; a0 += (int64_t)gridDim.x * kArcTile) {
    const int cnt = (int)(A - a0 < kArcTile ? A - a0 : kArcTile);
    const int64_t t = a0 / kArcTile;
    arc_tile_rows(off, n, a0, cnt, s_row, tile_row[t], tile_row[t + 1]);
    // Survivors are written warp-contiguously per unrolled step (order in
    // the list does not matter), so every store instruction is coalesced.
    // All label gathers of the tile are issued before the first hook atomic
    // (the atomics would otherwise order the next arc's gathers behind them).
    int32_t bu[kArcPer], bv[kArcPer];
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      bv[k] = i < cnt ? ld_stream(&col[a0 + i], once) : -1;
    }
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int i = k * kArcThreads + threadIdx.x;
      const int32_t v = bv[k];
      bu[k] = 0;
      bv[k] = 0;
      if (i < cnt) {
        const int32_t u = s_row[i];
        if (v < 0 || (int64_t)v >= n) {
          raise_error(status, DERR_INDEX);
        } else if (v > u) {
          bu[k] = C1[u];
          bv[k] = C1[v];
          mask |= 1u << k;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const int32_t cu = bu[k], cv = bv[k];
      if (((mask >> k) & 1u) && cu != cv) {
        // the first contraction round's hook, fused into the scan.  With
        // millions of slots contention is low, and reading a slot before its
        // atomic (as later rounds do) would only add a round trip here.
        const int i = k * kArcThreads + threadIdx.x;
        const unsigned long long key = (unsigned long long)(uint32_t)(a0 + i) << 32;
        const unsigned long long ku = key | (uint32_t)cv, kv = key | (uint32_t)cu;
        atomicMin(&best[cu], ku);
        atomicMin(&best[cv], kv);
      } else {
        mask &= ~(1u << k);
      }
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned wtot = 0;
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) wtot += __popc(__ballot_sync(0xffffffffu, (mask >> k) & 1u));
    const unsigned long long mine = block_reserve<kArcThreads>(counter, lane == 0 ? wtot : 0u);
    unsigned long long run = __shfl_sync(0xffffffffu, mine, 0);
#pragma unroll
    for (int k = 0; k < kArcPer; ++k) {
      const unsigned bal = __ballot_sync(0xffffffffu, (mask >> k) & 1u);
      if ((mask >> k) & 1u) {
        const unsigned long long slot = run + __popc(bal & lt);
        if ((int64_t)slot < cap) {
          Ecu[slot] = bu[k];
          Ecv[slot] = bv[k];
          Ep[slot] = (uint32_t)(a0 + k * kArcThreads + threadIdx.x);
        } else {
          raise_error(status, DERR_CAPACITY);
        }
      }
      run += __popc(bal);
    }
    __syncthreads();
  }
}

// k_build_list's grid: one tile per block up to this many blocks (the row
// searches of many resident blocks overlap); larger lists loop over tiles.
// Graphs with long rows take a smaller grid: there a giant round-1 component
// usually makes the kernel exit at once, and every launched block costs.
constexpr int64_t kListMaxBlocks = 1 << 16;
constexpr int64_t kListMaxBlocksLong = 1 << 12;

// tile_row for k_build_list (as k_arc_tile_rows), skipped when
// k_build_list_sparse builds the list.
template <class OffT>
__global__ void k_list_tile_rows(const OffT* __restrict__ off, int64_t n, int64_t A, int64_t tiles,
                                 int32_t* __restrict__ tile_row, const CcCtl* ctl) {
  pdl_wait();  // launched as a programmatic dependent
  if (sparse_list(ctl)) return;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t * kArcTile < A ? t * kArcTile : A - 1;
    tile_row[t] = (int32_t)row_of_arc(off, n, a < 0 ? 0 : a);
  }
}

// The same list and first hook when a giant round-1 component g exists, from
// the rows of the vertices outside it only: an inter-component edge has at
// least one end outside g.  Each warp takes 32 consecutive vertices and
// reads, together, the rows of those with edges outside g (ctl->ng counts
// them).  An edge between two such vertices is taken from its smaller end's
// row; an edge with one end in g from the outside end's row, its key (the
// position of the arc min -> max) found by a search of g's end's row when
// that end is the smaller one.
template <class OffT>
__global__ void __launch_bounds__(kBlock, 6) k_build_list_sparse(const OffT* __restrict__ off,
                                                              const int32_t* __restrict__ col, int64_t n,
                                                              const int32_t* __restrict__ C1, CcCtl* ctl,
                                                              unsigned long long* counter,
                                                              int32_t* __restrict__ Ecu, int32_t* __restrict__ Ecv,
                                                              uint32_t* __restrict__ Ep, int64_t cap,
                                                              unsigned long long* __restrict__ best,
                                                              uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  if (!sparse_list(ctl)) return;
  const int32_t cg = C1[ctl->giant];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned outside = 0;
  constexpr int kChunks = 4;  // 32-vertex chunks per warp and step, their labels read together
  for (int64_t w00 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 * kChunks); w00 < n;
       w00 += warps * (32 * kChunks)) {
    int32_t cls[kChunks];
#pragma unroll
    for (int k = 0; k < kChunks; ++k) {
      const int64_t v = w00 + 32 * k + lane;
      cls[k] = v < n ? C1[v] : -1;
    }
#pragma unroll
    for (int k = 0; k < kChunks; ++k) {
      const int32_t cl = cls[k];
      unsigned todo = __ballot_sync(0xffffffffu, cl >= 0 && cl != cg);
      outside += __popc(todo);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t u = (int32_t)(w00 + 32 * k + src);
        const int32_t cu = __shfl_sync(0xffffffffu, cl, src);
        const int64_t lo = (int64_t)off[u], hi = (int64_t)off[u + 1];
        for (int64_t a0 = lo; a0 < hi; a0 += 32) {
          const int64_t a = a0 + lane;
          bool emit = false;
          int32_t eu = 0, ev = 0;
          uint32_t p = 0;
          if (a < hi) {
            const int32_t x = col[a];
            if (x < 0 || (int64_t)x >= n) {
              raise_error(status, DERR_INDEX);
            } else if (x != u) {
              const int32_t cx = C1[x];
              if (cx < 0) {
                raise_error(status, DERR_INDEX);  // x has no arcs: the CSR is not symmetric
              } else if (cx != cu) {
                if (u < x) {
                  emit = true;
                  p = (uint32_t)a;
                  eu = cu;
                  ev = cx;
                } else if (cx == cg) {  // g's rows are not read: take the edge from this side
                  const int64_t q = row_find(off, col, x, u);
                  if (q < 0) {
                    raise_error(status, DERR_INDEX);
                  } else {
                    emit = true;
                    p = (uint32_t)q;
                    eu = cx;
                    ev = cu;
                  }
                }
              }
            }
          }
          if (emit) {  // the first contraction round's hook
            const unsigned long long key = (unsigned long long)p << 32;
            atomicMin(&best[eu], key | (uint32_t)ev);
            atomicMin(&best[ev], key | (uint32_t)eu);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, emit);
          unsigned long long at = 0;
          if (lane == 0 && bal) at = atomicAdd(counter, (unsigned long long)__popc(bal));
          at = __shfl_sync(0xffffffffu, at, 0);
          if (emit) {
            const unsigned long long slot = at + __popc(bal & lt);
            if ((int64_t)slot < cap) {
              Ecu[slot] = eu;
              Ecv[slot] = ev;
              Ep[slot] = p;
            } else {
              raise_error(status, DERR_CAPACITY);
            }
          }
        }
      }
    }
  }
  if (lane == 0 && outside) atomicAdd(&ctl->ng, outside);
}

// ------------------------------------------------------------------ rounds >= 2
//
// Round r on the contracted graph (components have dense ids 0..C-1):
//  1 hook: map every list entry through the previous round's component map,
//    drop entries inside one component, packed atomicMin on both endpoints,
//    and append the survivors (the next round's list)
//  2 resolve: final components, mutual pairs, hooks, tree-edge records
//  3 settle: shortcut the hook forest; dense ids for the surviving roots;
//    final components join the list of component roots
//  4 map: component -> next id; minimum vertex per new component; the last
//    block advances the round and sets the loop condition

// Once few components remain, every list entry hits one of a few hook slots;
// packed together they fall on a handful of L2 lines (and slices), which then
// serialise the atomics.  Rounds entering with at most kSpreadMaxC components
// give every slot its own 128-byte line when the buffer has room.
constexpr int kSpread = 16;
constexpr int64_t kSpreadMaxC = 1 << 16;
__device__ __forceinline__ int64_t next_round_stride(int64_t C, int64_t cap) {
  return (C <= kSpreadMaxC && C * kSpread <= cap) ? kSpread : 1;
}

struct CcPtrs {
  const int32_t* col;
  const RowRec* rec;  // row records (null: the twin is found by binary search)
  int32_t* Ecu[2];
  int32_t* Ecv[2];
  uint32_t* Ep[2];
  unsigned long long* best[2];
  int32_t* P2;
  int32_t* NID;
  int32_t* nextpool;
  int32_t* minvpool;
  uint4* pairs;
  uint32_t* bits;
  int32_t* roots;
  CcCtl* ctl;
  unsigned long long* counters;
  uint32_t* status;
  unsigned long long* tkey;
  uint32_t* tval;
  uint32_t* tp;
  int64_t ecap;
  int64_t bcap;  // slots in each best[] buffer
};

__global__ void __launch_bounds__(kBlock) k_round_init(CcPtrs b, int32_t root, const int32_t* __restrict__ C1,
                                                       int64_t n, const int32_t* __restrict__ P,
                                                       const uint32_t* __restrict__ J, int giant_pct) {
  pdl_wait();  // launched as a programmatic dependent
  if (blockIdx.x == 0) giant_sample(n, P, J, giant_pct, b.ctl);
  const unsigned long long C = b.counters[CNT_COMPS];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < (int64_t)C;
       c += (int64_t)gridDim.x * blockDim.x)
    b.best[0][c] = ~0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kTailSlots;
       i += (int64_t)gridDim.x * blockDim.x) {
    b.tkey[i] = ~0ull;  // the tail's pair table starts empty
    b.tval[i] = ~0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CcCtl* t = b.ctl;
    t->st[0].C = C;
    t->st[0].E = 0;  // the list build already hooked round 0; its list is round 1's
    t->st[0].pool_at = 0;
    t->st[0].bs = 1;
    const int32_t c1 = root >= 0 ? C1[root] : -1;
    t->st[0].rc = c1;
    t->root_label = (root >= 0 && c1 < 0) ? root : -1;
    t->cur = 0;
  }
}

// With at most kHookLocal components, entries first meet in a block-local
// copy of the hook slots (shared memory) and each block then offers one key
// per touched slot, instead of every entry contending on a few global slots.
constexpr int kHookLocal = 1024;
constexpr int kHookPer = 4;  // list entries per thread and step
constexpr int kHookBlocksPerSm = 6;  // resident at the register budget below
__global__ void __launch_bounds__(kBlock, kHookBlocksPerSm) k_round_hook(CcPtrs b) {
  __shared__ unsigned long long s_best[kHookLocal];
  CcCtl* t = b.ctl;
  const int r = t->cur;
  const int64_t E = (int64_t)t->st[r].E;
  const int64_t Cr = (int64_t)t->st[r].C;
  const bool local = Cr <= kHookLocal;
  if (local) {
    for (int c = threadIdx.x; c < Cr; c += blockDim.x) s_best[c] = ~0ull;
    __syncthreads();
  }
  const int src = r & 1, dst = src ^ 1;
  const int32_t* __restrict__ mp = r == 0 ? nullptr : b.nextpool + t->st[r - 1].pool_at;
  unsigned long long* __restrict__ best = b.best[r & 1];
  const int64_t bs = t->st[r].bs;
  const int32_t* __restrict__ Icu = b.Ecu[src];
  const int32_t* __restrict__ Icv = b.Ecv[src];
  const uint32_t* __restrict__ Ip = b.Ep[src];
  const int64_t tile = (int64_t)blockDim.x * kHookPer;
  const int64_t stride = (int64_t)gridDim.x * tile;
  const uint64_t once = l2_evict_first();  // this round's list is read once
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < E; base += stride) {
    // A thread takes kHookPer entries; all their reads and component-map
    // gathers are issued before the first hook atomic, so several chains of
    // dependent loads are in flight at once.
    int32_t cu[kHookPer], cv[kHookPer];
    uint32_t p[kHookPer];
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < kHookPer; ++k) {
      const int64_t e = base + (int64_t)k * blockDim.x + threadIdx.x;
      cu[k] = 0;
      cv[k] = 0;
      p[k] = 0;
      if (e < E) {
        cu[k] = ld_stream(&Icu[e], once);
        cv[k] = ld_stream(&Icv[e], once);
        p[k] = ld_stream(&Ip[e], once);
        mask |= 1u << k;
      }
    }
    if (mp) {
#pragma unroll
      for (int k = 0; k < kHookPer; ++k)
        if ((mask >> k) & 1u) {
          cu[k] = mp[cu[k]];
          cv[k] = mp[cv[k]];
        }
    }
#pragma unroll
    for (int k = 0; k < kHookPer; ++k)
      if (cu[k] == cv[k]) mask &= ~(1u << k);
    if (local) {
#pragma unroll
      for (int k = 0; k < kHookPer; ++k)
        if ((mask >> k) & 1u) {
          const unsigned long long key = (unsigned long long)p[k] << 32;
          atomicMin(&s_best[cu[k]], key | (uint32_t)cv[k]);
          atomicMin(&s_best[cv[k]], key | (uint32_t)cu[k]);
        }
    } else {
      // read before the atomic: a value already below the key (possibly
      // stale, values only decrease) makes the atomic unnecessary, which
      // removes most of the contention once few components remain
      unsigned long long ou[kHookPer], ov[kHookPer];
#pragma unroll
      for (int k = 0; k < kHookPer; ++k) {
        ou[k] = 0;
        ov[k] = 0;
        if ((mask >> k) & 1u) {
          ou[k] = __ldcg(&best[cu[k] * bs]);
          ov[k] = __ldcg(&best[cv[k] * bs]);
        }
      }
#pragma unroll
      for (int k = 0; k < kHookPer; ++k)
        if ((mask >> k) & 1u) {
          const unsigned long long key = (unsigned long long)p[k] << 32;
          const unsigned long long ku = key | (uint32_t)cv[k], kv = key | (uint32_t)cu[k];
          if (ou[k] > ku) atomicMin(&best[cu[k] * bs], ku);
          if (ov[k] > kv) atomicMin(&best[cv[k] * bs], kv);
        }
    }
    // survivors: one reservation per warp, written warp-contiguously per step
    unsigned wtot = 0;
#pragma unroll
    for (int k = 0; k < kHookPer; ++k) wtot += __popc(__ballot_sync(0xffffffffu, (mask >> k) & 1u));
    const unsigned long long mine = block_reserve<kBlock>(&t->st[r + 1].E, lane == 0 ? wtot : 0u);
    unsigned long long run = __shfl_sync(0xffffffffu, mine, 0);
#pragma unroll
    for (int k = 0; k < kHookPer; ++k) {
      const unsigned bal = __ballot_sync(0xffffffffu, (mask >> k) & 1u);
      if ((mask >> k) & 1u) {
        const unsigned long long slot = run + __popc(bal & lt);
        if ((int64_t)slot < b.ecap) {
          b.Ecu[dst][slot] = cu[k];
          b.Ecv[dst][slot] = cv[k];
          b.Ep[dst][slot] = p[k];
        } else {
          raise_error(b.status, DERR_CAPACITY);
        }
      }
      run += __popc(bal);
    }
  }
  if (local) {
    __syncthreads();
    for (int c = threadIdx.x; c < Cr; c += blockDim.x) {
      const unsigned long long k = s_best[c];
      unsigned long long* g = &best[c * bs];
      if (k != ~0ull && __ldcg(g) > k) atomicMin(g, k);
    }
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

// The same from b's row record when it holds the whole row: the entries below b
// (a < b: keys name arcs min -> max) are the candidates, and their row starts
// are read together instead of one binary-search step after another.
template <class OffT>
__device__ __forceinline__ bool twin_from_record(const OffT* __restrict__ off, const RowRec& R,
                                                 int32_t b, uint64_t p, int32_t* a_out, int64_t* q_out) {
  uint64_t lo[kRecCols], hi[kRecCols];
#pragma unroll
  for (int i = 0; i < kRecCols; ++i) {
    const bool cand = i < (int)R.deg && R.c[i] >= 0 && R.c[i] < b;
    lo[i] = cand ? (uint64_t)off[R.c[i]] : ~0ull;
    hi[i] = cand ? (uint64_t)off[R.c[i] + 1] : 0ull;
  }
  bool found = false;
#pragma unroll
  for (int i = 0; i < kRecCols; ++i)
    if (lo[i] <= p && p < hi[i]) {
      found = true;
      *a_out = R.c[i];
      *q_out = (int64_t)R.start + i;
    }
  return found;
}

// A component with no incident edge is final; otherwise it hooks onto the
// component its minimum-key edge reaches, except the smaller id of a mutual
// pair, which stays a root.  Each hook records its tree edge.
constexpr int kResolvePer = 2;  // components per thread and step
constexpr int kResolveBlocksPerSm = 5;
template <class OffT>
__global__ void __launch_bounds__(kBlock, kResolveBlocksPerSm) k_round_resolve(CcPtrs b, const OffT* __restrict__ off) {
  CcCtl* t = b.ctl;
  const int r = t->cur;
  const int64_t C = (int64_t)t->st[r].C;
  const unsigned long long* __restrict__ best = b.best[r & 1];
  const int64_t bs = t->st[r].bs;
  const int64_t tile = (int64_t)blockDim.x * kResolvePer;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < C; base += (int64_t)gridDim.x * tile) {
    // the slot, arc and partner reads of both components are in flight together
    unsigned long long bc[kResolvePer];
    int32_t bb[kResolvePer];
    uint32_t pk[kResolvePer];
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) {
      const int64_t c = base + (int64_t)j * blockDim.x + threadIdx.x;
      bc[j] = c < C ? best[c * bs] : ~0ull;
    }
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) {
      bb[j] = 0;
      pk[j] = 0;
      if (bc[j] != ~0ull) {
        bb[j] = b.col[(uint32_t)(bc[j] >> 32)];
        pk[j] = (uint32_t)(best[(int64_t)(uint32_t)(bc[j] & 0xffffffffull) * bs] >> 32);
      }
    }
    uint32_t hook = 0;
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) {
      const int64_t c = base + (int64_t)j * blockDim.x + threadIdx.x;
      if (c < C) {
        const int32_t c2 = (int32_t)(uint32_t)(bc[j] & 0xffffffffull);
        const uint32_t p = (uint32_t)(bc[j] >> 32);
        if (bc[j] == ~0ull || (pk[j] == p && (int32_t)c < c2)) {
          b.P2[c] = (int32_t)c;  // final, or the smaller end of a mutual pair
        } else {
          b.P2[c] = c2;
          hook |= 1u << j;
        }
      }
    }
    RowRec R[kResolvePer];
    if (b.rec) {
#pragma unroll
      for (int j = 0; j < kResolvePer; ++j)
        if ((hook >> j) & 1u) R[j] = b.rec[bb[j]];
    }
    uint4 out[kResolvePer];
    uint32_t emit = 0;
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) {
      out[j] = make_uint4(0, 0, 0, 0);
      if ((hook >> j) & 1u) {
        const uint32_t p = (uint32_t)(bc[j] >> 32);
        int32_t a = 0;
        int64_t q = 0;
        bool found;
        if (b.rec && R[j].deg <= (uint32_t)kRecCols)
          found = twin_from_record(off, R[j], bb[j], (uint64_t)p, &a, &q);
        else
          found = twin_of_position(off, b.col, bb[j], (uint64_t)p, &a, &q);
        if (found) {
          emit |= 1u << j;
          out[j] = make_uint4(p, (uint32_t)q, (uint32_t)a, (uint32_t)bb[j]);
        } else {
          raise_error(b.status, DERR_INDEX);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j)
      if ((emit >> j) & 1u) {
        atomicOr(&b.bits[out[j].x >> 5], 1u << (out[j].x & 31));
        atomicOr(&b.bits[out[j].y >> 5], 1u << (out[j].y & 31));
      }
    unsigned wtot = 0;
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) wtot += __popc(__ballot_sync(0xffffffffu, (emit >> j) & 1u));
    const unsigned long long mine = block_reserve<kBlock>(&b.counters[CNT_PAIRS], lane == 0 ? wtot : 0u);
    unsigned long long run = __shfl_sync(0xffffffffu, mine, 0);
#pragma unroll
    for (int j = 0; j < kResolvePer; ++j) {
      const unsigned bal = __ballot_sync(0xffffffffu, (emit >> j) & 1u);
      if ((emit >> j) & 1u) b.pairs[run + __popc(bal & lt)] = out[j];
      run += __popc(bal);
    }
  }
}

// Pointer jumping over the component forest (every component shortcut to its
// root, in place: only thread c writes P2[c], and any value another thread
// reads is an ancestor), and dense ids for the roots that still have edges
// (their next-round hook slot starts empty and their minimum vertex starts as
// their own); components without edges are final and their minimum vertex
// joins the root list.  Roots are fixed points, so the root test does not
// depend on the shortcut.
__global__ void k_round_settle(CcPtrs b) {
  CcCtl* t = b.ctl;
  const int r = t->cur;
  const int64_t C = (int64_t)t->st[r].C;
  const unsigned long long* __restrict__ best = b.best[r & 1];
  unsigned long long* __restrict__ best_next = b.best[(r + 1) & 1];
  const int64_t bs = t->st[r].bs, bsn = next_round_stride(C, b.bcap);
  const int32_t* __restrict__ minv = b.minvpool + t->st[r].pool_at;
  int32_t* __restrict__ minv_next = b.minvpool + t->st[r].pool_at + C;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < C; base += stride) {
    const int64_t c = base + threadIdx.x;
    bool live_root = false, fin = false;
    if (c < C) {
      fin = best[c * bs] == ~0ull;
      int32_t x = b.P2[c];
      live_root = !fin && x == (int32_t)c;
      int64_t it = 0;
      while (true) {
        const int32_t y = b.P2[x];
        if (y == x) break;
        x = y;
        if (++it > C) {
          raise_error(b.status, DERR_ROUND_LIMIT);
          break;
        }
      }
      b.P2[c] = x;
    }
    const unsigned long long id = block_reserve<kBlock>(&t->st[r + 1].C, live_root ? 1u : 0u);
    const unsigned long long rid = block_reserve<kBlock>(&b.counters[CNT_ROOTS], fin ? 1u : 0u);
    if (c < C) b.NID[c] = live_root ? (int32_t)id : -1;
    if (fin) b.roots[rid] = minv[c];
    if (live_root) {
      best_next[(int64_t)id * bsn] = ~0ull;
      minv_next[id] = minv[c];
    }
  }
}

// Component -> next id and minimum vertex per new component.  The last block
// to finish advances the round and sets the loop condition (no separate
// kernel; every block has read the round index before it counts itself done).
__global__ void k_round_map(CcPtrs b, cudaGraphConditionalHandle h, int use_handle, int allow_tail) {
  CcCtl* t = b.ctl;
  const int r = t->cur;
  const int64_t C = (int64_t)t->st[r].C;
  const unsigned long long* __restrict__ best = b.best[r & 1];
  const int32_t* __restrict__ minv = b.minvpool + t->st[r].pool_at;
  int32_t* __restrict__ minv_next = b.minvpool + t->st[r].pool_at + C;
  int32_t* __restrict__ next = b.nextpool + t->st[r].pool_at;
  const int rc = t->st[r].rc;
  const int64_t bs = t->st[r].bs;
  // blocks past the work neither map nor count themselves done
  const int64_t want = (C + blockDim.x - 1) / blockDim.x;
  const unsigned nb = want < 1 ? 1u : (want < (int64_t)gridDim.x ? (unsigned)want : gridDim.x);
  if (blockIdx.x >= nb) return;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    const bool fin = best[c * bs] == ~0ull;
    int32_t nc = kFinal;
    if (!fin) {
      const int32_t root = b.P2[c];
      nc = b.NID[root];
      if (root != (int32_t)c) atomicMin(&minv_next[nc], minv[c]);
    }
    next[c] = nc;
    if ((int32_t)c == rc) {
      t->st[r + 1].rc = nc;
      if (fin) t->root_label = minv[c];
    }
  }
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&t->done, 1u) == nb - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    t->done = 0;
    t->st[r + 1].pool_at = t->st[r].pool_at + C;
    t->st[r + 1].bs = (int)next_round_stride(C, b.bcap);
    if (rc < 0) t->st[r + 1].rc = -1;
    const int nr = r + 1;
    bool more = t->st[nr].C > 0;
    if (more && nr >= kMaxRounds) {
      raise_error(b.status, DERR_ROUND_LIMIT);
      more = false;
    }
    if (more && allow_tail && t->st[nr].C <= (unsigned long long)kTailC) {
      t->tail = 1;  // the tail takes the remaining rounds
      t->tail_round = nr;
      more = false;
    }
    t->cur = nr;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
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

// ------------------------------------------------------------------ the tail

// One entry per component pair of the list entering round tail_round: the
// pair's smallest key (Fibonacci hashing, linear probing in an L2-resident
// table; a full probe sequence flags an overflow and the tail is not run).
__global__ void k_tail_dedup(CcPtrs b) {
  CcCtl* t = b.ctl;
  if (t->tail != 1) return;
  const int R = t->tail_round;
  const int64_t E = (int64_t)t->st[R].E;
  const int src = R & 1;
  const int32_t* __restrict__ mp = b.nextpool + t->st[R - 1].pool_at;
  const int32_t* __restrict__ Icu = b.Ecu[src];
  const int32_t* __restrict__ Icv = b.Ecv[src];
  const uint32_t* __restrict__ Ip = b.Ep[src];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    // once the table has overflowed the tail will not run: stop early
    if (__ldcg(&t->tail_overflow) != 0u) break;
    const int32_t cu = mp[Icu[e]], cv = mp[Icv[e]];
    if (cu == cv || cu < 0 || cv < 0) continue;
    const uint32_t p = Ip[e];
    const unsigned long long key = cu < cv ? ((unsigned long long)(uint32_t)cu << 32) | (uint32_t)cv
                                           : ((unsigned long long)(uint32_t)cv << 32) | (uint32_t)cu;
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - kTailBits));
    bool placed = false;
    for (int probe = 0; probe < kTailProbe; ++probe) {
      unsigned long long old = __ldcg(&b.tkey[h]);
      if (old == ~0ull) old = atomicCAS(&b.tkey[h], ~0ull, key);
      if (old == ~0ull || old == key) {
        if (__ldcg(&b.tval[h]) > p) atomicMin(&b.tval[h], p);
        placed = true;
        break;
      }
      h = (h + 1) & (kTailSlots - 1);
    }
    if (!placed) atomicExch(&t->tail_overflow, 1u);
  }
}

// Exclusive prefix sum over the block (kTailThreads threads); *total = sum.
__device__ __forceinline__ int tail_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    int ws = w;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ws, d);
      if (lane >= d) ws += y;
    }
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = ws - w;
    if (lane == 31) s_warp[32] = ws;
  }
  __syncthreads();
  const int r = x - v + s_warp[warp];
  *total = s_warp[32];
  __syncthreads();
  return r;
}

// All remaining rounds in one block, on the deduplicated pairs: the same
// hooking, mutual-pair rule, tree-edge choice, compression and minimum
// vertices as the regular rounds.  Final components join the root list as
// they appear; the final label of every component entering the tail is
// written over its minimum vertex (the labels pass reads it as the last
// round's labels); the tree edges' keys go to tp for k_tail_records.
__global__ void __launch_bounds__(kTailThreads) k_tail(CcPtrs b, cudaGraphConditionalHandle h2, int use_handle) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* s_best = reinterpret_cast<unsigned long long*>(smem);  // kTailC
  int32_t* s_par = reinterpret_cast<int32_t*>(s_best + kTailC);             // parent, then next id
  int32_t* s_minv = s_par + kTailC;
  int32_t* s_minv2 = s_minv + kTailC;
  int32_t* s_nid = s_minv2 + kTailC;  // -1 final, -2 hooked, else the live root's next id
  int32_t* s_cur = s_nid + kTailC;    // entering component x: its current component (-1: done)
  int32_t* s_lab = s_cur + kTailC;    // entering component x: its final label
  uint32_t* s_pu = reinterpret_cast<uint32_t*>(s_lab + kTailC);  // kTailPairs
  uint32_t* s_pv = s_pu + kTailPairs;
  uint32_t* s_pp = s_pv + kTailPairs;
  __shared__ int s_warp[33];
  __shared__ int s_np, s_bad, s_hooks, s_flag, s_rc;
  CcCtl* t = b.ctl;
  if (t->tail != 1) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int R = t->tail_round;
  const int C0 = (int)t->st[R].C;
  if (tid == 0) {
    s_np = 0;
    s_bad = (t->tail_overflow != 0u || C0 > kTailC) ? 1 : 0;
    s_hooks = 0;
    s_rc = t->st[R].rc;
  }
  __syncthreads();
  if (!s_bad) {
    // the table's pairs into shared memory, one position reservation per
    // warp and step (kTailSlots is a multiple of the block size)
    for (int s0 = 0; s0 < kTailSlots; s0 += nt) {
      const int slot = s0 + tid;
      const unsigned long long key = b.tkey[slot];
      const bool has = key != ~0ull;
      const unsigned bal = __ballot_sync(0xffffffffu, has);
      int at = 0;
      if ((tid & 31) == 0 && bal) at = atomicAdd(&s_np, __popc(bal));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (has) {
        const int i = at + __popc(bal & ((1u << (tid & 31)) - 1u));
        if (i < kTailPairs) {
          s_pu[i] = (uint32_t)(key >> 32);
          s_pv[i] = (uint32_t)(key & 0xffffffffull);
          s_pp[i] = b.tval[slot];
        } else {
          s_bad = 1;
        }
      }
    }
  }
  __syncthreads();
  if (s_bad) {  // does not fit: the regular rounds continue from round R
    for (int slot = tid; slot < kTailSlots; slot += nt) {  // empty table for the next request
      b.tkey[slot] = ~0ull;
      b.tval[slot] = ~0u;
    }
    if (tid == 0) {
      t->tail = 3;
      t->tail_overflow = 0u;
      if (t->tail_backs++ == 0) t->tail_first_back = R;
      if (use_handle) cudaGraphSetConditional(h2, 1u);
    }
    return;
  }
  const int32_t* __restrict__ minv_in = b.minvpool + t->st[R].pool_at;
  for (int c = tid; c < C0; c += nt) {
    s_minv[c] = minv_in[c];
    s_cur[c] = c;
    s_lab[c] = -1;
  }
  int C = C0, np = s_np;
  int rounds = 0;
  bool converged = false;
  for (; rounds < kTailMaxRounds; ++rounds) {
    for (int c = tid; c < C; c += nt) s_best[c] = ~0ull;
    __syncthreads();
    for (int i = tid; i < np; i += nt) {
      // read before the atomic: slot values only fall, so most atomics are skipped
      const unsigned long long key = (unsigned long long)s_pp[i] << 32;
      const unsigned long long ku = key | s_pv[i], kv = key | s_pu[i];
      if (s_best[s_pu[i]] > ku) atomicMin(&s_best[s_pu[i]], ku);
      if (s_best[s_pv[i]] > kv) atomicMin(&s_best[s_pv[i]], kv);
    }
    __syncthreads();
    for (int c0 = 0; c0 < C; c0 += nt) {  // resolve (every lane of a warp takes each step)
      const int c = c0 + tid;
      bool hook = false;
      uint32_t p = 0;
      if (c < C) {
        const unsigned long long bc = s_best[c];
        if (bc == ~0ull) {
          s_par[c] = c;
          s_nid[c] = -1;
        } else {
          const int c2 = (int)(bc & 0xffffffffull);
          p = (uint32_t)(bc >> 32);
          if ((uint32_t)(s_best[c2] >> 32) == p && c < c2) {
            s_par[c] = c;
            s_nid[c] = 0;
          } else {
            s_par[c] = c2;
            s_nid[c] = -2;
            hook = true;
          }
        }
      }
      // one slot reservation per warp (a single shared counter serialises
      // per-thread atomics); fewer than C0 <= kTailC hooks in all
      const unsigned bal = __ballot_sync(0xffffffffu, hook);
      int at = 0;
      if ((tid & 31) == 0 && bal) at = atomicAdd(&s_hooks, __popc(bal));
      at = __shfl_sync(0xffffffffu, at, 0);
      if (hook) b.tp[at + __popc(bal & ((1u << (tid & 31)) - 1u))] = p;
    }
    __syncthreads();
    for (int it = 0; it < 32; ++it) {  // compress (pointer jumping in place)
      if (tid == 0) s_flag = 0;
      __syncthreads();
      for (int c = tid; c < C; c += nt) {
        const int x = s_par[c], y = s_par[x];
        if (y != x) {
          s_par[c] = y;
          s_flag = 1;
        }
      }
      __syncthreads();
      const int f = s_flag;
      __syncthreads();
      if (!f) break;
      if (it == 31 && tid == 0) raise_error(b.status, DERR_ROUND_LIMIT);
    }
    // next ids of live roots, in component order; final components leave
    int base = 0;
    for (int c0 = 0; c0 < C; c0 += nt) {
      const int c = c0 + tid;
      const int live = (c < C && s_nid[c] == 0) ? 1 : 0;
      int tot = 0;
      const int ex = tail_scan(live, s_warp, &tot);
      if (live) s_nid[c] = base + ex;
      base += tot;
    }
    for (int c = tid; c < C; c += nt) {
      if (s_nid[c] == -1) {
        const unsigned long long rid = atomicAdd(&b.counters[CNT_ROOTS], 1ull);
        b.roots[rid] = s_minv[c];
        if (c == s_rc) t->root_label = s_minv[c];
      } else if (s_par[c] == c) {
        s_minv2[s_nid[c]] = s_minv[c];
      }
    }
    __syncthreads();
    for (int c = tid; c < C; c += nt) {  // next id of every component (-1: final)
      int nx = s_nid[c] == -1 ? -1 : s_nid[s_par[c]];
      if (s_nid[c] == -2) {
        if (nx >= 0 && nx < base) {
          atomicMin(&s_minv2[nx], s_minv[c]);
        } else {  // a hooked component whose root is not live: cannot happen
          raise_error(b.status, DERR_INDEX);
          nx = -1;
        }
      }
      s_par[c] = nx;
    }
    __syncthreads();
    if (tid == 0) s_rc = s_rc >= 0 ? s_par[s_rc] : -1;
    for (int x = tid; x < C0; x += nt) {  // the entering components' labels
      const int c = s_cur[x];
      if (c < 0) continue;
      if (s_nid[c] == -1) {
        s_lab[x] = s_minv[c];
        s_cur[x] = -1;
      } else {
        s_cur[x] = s_par[c];
      }
    }
    // the pairs in next ids, without those inside one component
    constexpr int kPer = kTailPairs / kTailThreads;
    static_assert(kPer * kTailThreads == kTailPairs, "pairs must split evenly over the block");
    uint32_t u[kPer], v[kPer], pp[kPer];
    int keep = 0;
    for (int k = 0; k < kPer; ++k) {
      const int i = k * nt + tid;
      u[k] = v[k] = pp[k] = 0;
      if (i < np) {
        u[k] = (uint32_t)s_par[s_pu[i]];
        v[k] = (uint32_t)s_par[s_pv[i]];
        pp[k] = s_pp[i];
        if (u[k] != v[k]) {
          if (u[k] < (uint32_t)base && v[k] < (uint32_t)base)
            keep |= 1 << k;
          else  // an endpoint left as final while the pair remains: cannot happen
            raise_error(b.status, DERR_INDEX);
        }
      }
    }
    int tot = 0;
    int at = tail_scan(__popc(keep), s_warp, &tot);  // all reads of the old pairs are done
    for (int k = 0; k < kPer; ++k)
      if ((keep >> k) & 1) {
        s_pu[at] = u[k];
        s_pv[at] = v[k];
        s_pp[at] = pp[k];
        ++at;
      }
    for (int c = tid; c < base; c += nt) s_minv[c] = s_minv2[c];
    __syncthreads();
    C = base;
    np = tot;
    if (C == 0) {
      converged = true;
      ++rounds;
      break;
    }
  }
  if (!converged && tid == 0) raise_error(b.status, DERR_ROUND_LIMIT);
  int32_t* lab_out = b.minvpool + t->st[R].pool_at;
  for (int x = tid; x < C0; x += nt) lab_out[x] = s_lab[x];
  if (tid == 0) {
    t->tail_rounds = rounds;
    t->tail_hooks = (unsigned int)s_hooks;
    t->tail = 2;
  }
}

// The tail's tree edges as records {p, q, a, b} with both arcs marked, as
// k_round_resolve writes them (the twin found from b's row record or row).
template <class OffT>
__global__ void __launch_bounds__(kBlock) k_tail_records(CcPtrs b, const OffT* __restrict__ off) {
  CcCtl* t = b.ctl;
  if (t->tail != 2) return;
  const int64_t H = (int64_t)t->tail_hooks;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < H; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = base + threadIdx.x;
    bool emit = false;
    uint4 out = make_uint4(0, 0, 0, 0);
    if (j < H) {
      const uint32_t p = b.tp[j];
      const int32_t bb = b.col[p];
      int32_t a = 0;
      int64_t q = 0;
      bool found;
      if (b.rec) {
        const RowRec Rr = b.rec[bb];
        found = Rr.deg <= (uint32_t)kRecCols ? twin_from_record(off, Rr, bb, (uint64_t)p, &a, &q)
                                             : twin_of_position(off, b.col, bb, (uint64_t)p, &a, &q);
      } else {
        found = twin_of_position(off, b.col, bb, (uint64_t)p, &a, &q);
      }
      if (found) {
        emit = true;
        out = make_uint4(p, (uint32_t)q, (uint32_t)a, (uint32_t)bb);
        atomicOr(&b.bits[out.x >> 5], 1u << (out.x & 31));
        atomicOr(&b.bits[out.y >> 5], 1u << (out.y & 31));
      } else {
        raise_error(b.status, DERR_INDEX);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, emit);
    const unsigned long long mine = block_reserve<kBlock>(&b.counters[CNT_PAIRS], lane == 0 ? (unsigned)__popc(bal) : 0u);
    const unsigned long long w0 = __shfl_sync(0xffffffffu, mine, 0);
    if (emit) b.pairs[w0 + __popc(bal & lt)] = out;
  }
}

// ------------------------------------------------------------------ round graph

// One instantiated graph per (workspace, graph, round grid) binding: a
// while-conditional node whose body is the four round kernels.
struct RoundGraph {
  bool valid = false;
  const void* key_off = nullptr;
  const void* key_col = nullptr;
  const void* key_ws = nullptr;
  int64_t key_n = 0, key_A = 0;
  int key_dev = -1;
  int key_grid = 0;
  cudaGraphExec_t exec = nullptr;
};
constexpr int kGraphCache = 8;
static RoundGraph g_round_graphs[kGraphCache];
static int g_round_graph_next = 0;
static cudaStream_t g_capture_stream[64] = {};

void destroy_round_graphs() {
  for (auto& g : g_round_graphs) {
    if (g.valid && g.exec) cudaGraphExecDestroy(g.exec);
    g = RoundGraph{};
  }
}

template <class OffT>
static void launch_round_body(const CcPtrs& p, const OffT* off, cudaGraphConditionalHandle h,
                              int use_handle, int allow_tail, cudaStream_t s) {
  const int g = device_info().sms * tuning().round_bps;
  const int gh = device_info().sms * std::min(tuning().round_bps, kHookBlocksPerSm);
  // stage marks only where the rounds are stepped from the host (a mark is an
  // event, which a graph body captured here must not hold)
  RST_LAUNCH(k_round_hook, gh, kBlock, 0, s)(p);
  if (!use_handle) prof_mark(s, "rd_hook");
  const int gr = device_info().sms * std::min(tuning().round_bps, kResolveBlocksPerSm);
  RST_LAUNCH(k_round_resolve<OffT>, gr, kBlock, 0, s)(p, off);
  if (!use_handle) prof_mark(s, "rd_resolve");
  RST_LAUNCH(k_round_settle, g, kBlock, 0, s)(p);
  if (!use_handle) prof_mark(s, "rd_settle");
  RST_LAUNCH(k_round_map, g, kBlock, 0, s)(p, h, use_handle, allow_tail);
  if (!use_handle) prof_mark(s, "rd_map");
}

template <class OffT>
static void launch_tail(const CcPtrs& p, const OffT* off, cudaGraphConditionalHandle h2, int use_handle,
                        cudaStream_t s) {
  RST_LAUNCH(k_tail_dedup, device_info().sms * 8, kBlock, 0, s)(p);
  if (!use_handle) prof_mark(s, "tail_dedup");
  RST_LAUNCH(k_tail, 1, kTailThreads, kTailSmem, s)(p, h2, use_handle);
  if (!use_handle) prof_mark(s, "tail_rounds");
  RST_LAUNCH(k_tail_records<OffT>, device_info().sms * 4, kBlock, 0, s)(p, off);
  if (!use_handle) prof_mark(s, "tail_records");
}

// A while node whose body is one contraction round (captured from the
// round kernels), followed by the tail's kernels when with_tail is set,
// after the given dependencies.
template <class OffT>
static rst_status add_round_loop(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                                 cudaGraphConditionalHandle h, const CcPtrs& p, const OffT* off, bool with_tail,
                                 cudaStream_t cs, cudaGraphNode_t* node) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  RST_CUDA(cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  RST_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_round_body<OffT>(p, off, h, 1, 1, cs);
  if (with_tail) launch_tail<OffT>(p, off, h, 1, cs);
  cudaGraph_t captured = nullptr;
  RST_CUDA(cudaStreamEndCapture(cs, &captured));
  return RST_OK;
}

// Shared memory beyond the default for the tail's single block (once per device).
static rst_status tail_smem_attr() {
  static bool set[64] = {};
  int dev = 0;
  RST_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && set[dev]) return RST_OK;
  RST_CUDA(cudaFuncSetAttribute((const void*)k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTailSmem));
  if (dev >= 0 && dev < 64) set[dev] = true;
  return RST_OK;
}


template <class OffT>
static rst_status round_graph_for(const CcPtrs& p, const OffT* off, int64_t n, int64_t A,
                                  cudaGraphExec_t* out) {
  int dev = 0;
  RST_CUDA(cudaGetDevice(&dev));
  for (auto& g : g_round_graphs) {
    if (g.valid && g.key_off == off && g.key_col == p.col && g.key_ws == (const void*)p.ctl &&
        g.key_n == n && g.key_A == A && g.key_dev == dev && g.key_grid == tuning().round_bps) {
      *out = g.exec;
      return RST_OK;
    }
  }
  if (dev < 0 || dev >= 64) return RST_ERR_UNSUPPORTED;
  if (!g_capture_stream[dev])
    RST_CUDA(cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking));
  RST_TRY(tail_smem_attr());
  cudaStream_t cs = g_capture_stream[dev];
  // regular rounds (a while loop) -> the tail's three kernels -> a second
  // while loop of rounds each followed by the tail's kernels, entered only
  // when the tail hands back
  cudaGraph_t graph = nullptr;
  RST_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h1, h2;
  RST_CUDA(cudaGraphConditionalHandleCreate(&h1, graph, 1, cudaGraphCondAssignDefault));
  RST_CUDA(cudaGraphConditionalHandleCreate(&h2, graph, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t loop1, dedup, tailn, recs, loop2;
  RST_TRY(add_round_loop<OffT>(graph, nullptr, 0, h1, p, off, false, cs, &loop1));
  CcPtrs pc = p;
  int one = 1;
  void* dedup_args[] = {&pc};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_tail_dedup;
  kp.gridDim = dim3(device_info().sms * 8);
  kp.blockDim = dim3(kBlock);
  kp.kernelParams = dedup_args;
  RST_CUDA(cudaGraphAddKernelNode(&dedup, graph, &loop1, 1, &kp));
  void* tail_args[] = {&pc, &h2, &one};
  kp.func = (void*)k_tail;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kTailThreads);
  kp.sharedMemBytes = (unsigned)kTailSmem;
  kp.kernelParams = tail_args;
  RST_CUDA(cudaGraphAddKernelNode(&tailn, graph, &dedup, 1, &kp));
  const OffT* offp = off;
  void* rec_args[] = {&pc, &offp};
  kp.func = (void*)k_tail_records<OffT>;
  kp.gridDim = dim3(device_info().sms * 4);
  kp.blockDim = dim3(kBlock);
  kp.sharedMemBytes = 0;
  kp.kernelParams = rec_args;
  RST_CUDA(cudaGraphAddKernelNode(&recs, graph, &tailn, 1, &kp));
  RST_TRY(add_round_loop<OffT>(graph, &recs, 1, h2, p, off, true, cs, &loop2));
  cudaGraphExec_t exec = nullptr;
  RST_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  RST_CUDA(cudaGraphDestroy(graph));
  RoundGraph& slot = g_round_graphs[g_round_graph_next];
  g_round_graph_next = (g_round_graph_next + 1) % kGraphCache;
  if (slot.valid && slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.valid = true;
  slot.key_off = off;
  slot.key_col = p.col;
  slot.key_ws = p.ctl;
  slot.key_n = n;
  slot.key_A = A;
  slot.key_dev = dev;
  slot.key_grid = tuning().round_bps;
  slot.exec = exec;
  *out = exec;
  return RST_OK;
}

// ------------------------------------------------------------------ driver

template <class OffT>
rst_status cc_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A,
                  int32_t root, int32_t* labels_out, CcOut* out, cudaStream_t s, bool prefetch_euler) {
  CcBuffers b = cc_layout(ar, n, A);
  if (ar.used > ar.cap) return RST_ERR_OOM;  // some buffer of the layout did not fit (null)
  // Euler-stage buffers taken here when its first steps are queued early
  // (the Euler stage then takes them no more, so the total is unchanged)
  const int64_t W = A / 32 + 1;
  uint2* pre_rk = nullptr;
  unsigned long long* pre_tmp = nullptr;
  uint32_t* pre_root = nullptr;
  uint32_t* pre_rs = nullptr;
  if (prefetch_euler && state().readback && !state_overridden()) {
    pre_rk = ar.take<uint2>(W + 1);
    pre_tmp = ar.take<unsigned long long>(scan_tmp_words(W));
    pre_root = ar.take<uint32_t>(n / 32 + 1);
    pre_rs = ar.take<uint32_t>(row_start_words(A));
    if (!pre_rk || !pre_tmp || !pre_root || !pre_rs) return RST_ERR_OOM;
  }
  uint32_t* status = state().status;
  unsigned long long* cnt = dev_counter(0);
  RST_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  RST_CUDA(cudaMemsetAsync(b.bits, 0, (A / 32 + 2) * sizeof(uint32_t), s));
  RST_CUDA(cudaMemsetAsync(b.ctl, 0, sizeof(CcCtl), s));
  RST_CUDA(cudaMemsetAsync(b.rbits, 0, (n / 32 + 2) * sizeof(uint32_t), s));
  if (pre_rs) RST_CUDA(cudaMemsetAsync(pre_rs, 0, row_start_words(A) * sizeof(uint32_t), s));

  const int gN = grid_for(n);
  prof_mark(s, "cc_setup");
  RST_LAUNCH_PDL((k_r1_choose<OffT>), gN, kBlock, 0, s)(off, col, n, b.P, b.J, b.rec, pre_rs, status);
  prof_mark(s, "k_r1_choose");
  if (A > kR1LongRowDegree * n)
    RST_LAUNCH_PDL((k_r1_resolve<OffT, kR1PerLong, kR1BlocksPerSmLong>),
                   grid_for((n + kR1PerLong - 1) / kR1PerLong, kBlock, kR1BlocksPerSmLong), kBlock, 0, s)(
        off, col, n, b.P, b.J, b.rec, b.pairs, b.bits, b.rbits, cnt, status);
  else
    RST_LAUNCH_PDL((k_r1_resolve<OffT, kR1Per, kR1BlocksPerSm>), grid_for((n + kR1Per - 1) / kR1Per, kBlock, kR1BlocksPerSm),
                   kBlock, 0, s)(off, col, n, b.P, b.J, b.rec, b.pairs, b.bits, b.rbits, cnt, status);
  prof_mark(s, "k_r1_resolve");
  RST_TRY(scan_popcount_ranked(b.rbits, b.rrank, n / 32 + 1, b.rtmp, s));
  prof_mark(s, "r1_rootscan");
  RST_LAUNCH_PDL(k_r1_label, gN, kBlock, 0, s)(n, b.P, b.J, b.rrank, b.C1, b.minvpool, cnt);
  prof_mark(s, "k_r1_label");
  CcPtrs p;
  p.col = col;
  p.rec = b.rec;
  for (int k = 0; k < 2; ++k) {
    p.Ecu[k] = b.Ecu[k];
    p.Ecv[k] = b.Ecv[k];
    p.Ep[k] = b.Ep[k];
    p.best[k] = b.best[k];
  }
  p.P2 = b.P2;
  p.NID = b.NID;
  p.nextpool = b.nextpool;
  p.minvpool = b.minvpool;
  p.pairs = b.pairs;
  p.bits = b.bits;
  p.roots = b.roots;
  p.ctl = b.ctl;
  p.counters = cnt;
  p.status = status;
  p.tkey = b.tkey;
  p.tval = b.tval;
  p.tp = b.tp;
  p.ecap = b.ecap;
  p.bcap = b.bcap;
  RST_LAUNCH_PDL(k_round_init, grid_for(n / 2 + 1), kBlock, 0, s)(p, root, b.C1, A > 0 ? n : 0, b.P, b.J,
                                                                  tuning().giant_pct);
  prof_mark(s, "k_round_init");
  if (A > 0) {
    // one tile per block: the row searches of many resident blocks overlap;
    // entries go to list buffer 1 (round 1 reads it) and are counted in st[1].E
    const int64_t tiles = (A + kArcTile - 1) / kArcTile;
    const unsigned g = (unsigned)std::min<int64_t>(tiles, A > kR1LongRowDegree * n ? kListMaxBlocksLong : kListMaxBlocks);
    RST_LAUNCH_PDL((k_list_tile_rows<OffT>), grid_for(tiles + 1), kBlock, 0, s)(off, n, A, tiles, b.tile_row,
                                                                               b.ctl);
    RST_LAUNCH_PDL((k_build_list<OffT>), g, kArcThreads, 0, s)(off, col, n, A, b.C1, b.Ecu[1], b.Ecv[1],
                                                         b.Ep[1], &b.ctl->st[1].E, b.ecap, b.tile_row,
                                                         b.best[0], b.ctl, status);
    RST_LAUNCH_PDL((k_build_list_sparse<OffT>), grid_for(n, kBlock, 6), kBlock, 0, s)(
        off, col, n, b.C1, b.ctl, &b.ctl->st[1].E, b.Ecu[1], b.Ecv[1], b.Ep[1], b.ecap, b.best[0], status);
  }
  prof_mark(s, "k_build_list");
  RST_CUDA(cudaGetLastError());

  // Contraction rounds: one graph launch (a device-side while loop), or,
  // when this call must not allocate (no graph objects) or RST_EAGER is set,
  // a host loop that reads the component count after every round.
  static const bool eager_env = getenv("RST_EAGER") != nullptr;
  const bool eager = eager_env || state_overridden();
  if (!eager) {
    cudaGraphExec_t exec = nullptr;
    RST_TRY(round_graph_for<OffT>(p, off, n, A, &exec));
    RST_CUDA(cudaGraphLaunch(exec, s));
  } else {
    RST_TRY(tail_smem_attr());
    for (int r = 0; r < kMaxRounds; ++r) {
      launch_round_body<OffT>(p, off, cudaGraphConditionalHandle{}, 0, 1, s);
      RST_CUDA(cudaGetLastError());
      unsigned long long c = 0;
      RST_TRY(fetch_u64(&b.ctl->st[r + 1].C, 1, &c, s));
      if (c == 0) break;
      if (c <= (unsigned long long)kTailC && r + 1 < kMaxRounds) {
        // the device requested the tail (the same test as k_round_map's)
        launch_tail<OffT>(p, off, cudaGraphConditionalHandle{}, 0, s);
        RST_CUDA(cudaGetLastError());
        unsigned long long w = 0;  // tail (low half), tail_round (high half)
        RST_TRY(fetch_u64(reinterpret_cast<const unsigned long long*>(&b.ctl->tail), 1, &w, s));
        if ((int)(w & 0xffffffffull) == 2) break;
        // handed back: the regular rounds continue and request it again
      }
    }
  }
  prof_mark(s, "cc_rounds");

  // one read-back of the counters and the round control (pinned), with the
  // Euler stage's first steps queued behind it when requested
  static_assert(8 * sizeof(unsigned long long) + sizeof(CcCtl) <= kHostBufWords * sizeof(unsigned long long),
                "read-back buffer too small");
  unsigned long long* hb = state().hostbuf;
  CcCtl* hctl = reinterpret_cast<CcCtl*>(hb + 8);
  RST_CUDA(cudaMemcpyAsync(hb, cnt, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaMemcpyAsync(hctl, b.ctl, sizeof(CcCtl), cudaMemcpyDeviceToHost, s));
  if (pre_rk) {
    RST_CUDA(cudaEventRecord(state().readback, s));
    RST_TRY(scan_popcount_ranked(b.bits, pre_rk, W, pre_tmp, s));
    RST_CUDA(cudaMemsetAsync(pre_root, 0, (n / 32 + 1) * sizeof(uint32_t), s));
    RST_CUDA(cudaEventSynchronize(state().readback));
  } else {
    RST_CUDA(cudaStreamSynchronize(s));
  }
  unsigned long long h[8];
  for (int i = 0; i < 8; ++i) h[i] = hb[i];
  // with the tail, the labels of the components entering round tail_round
  // are final (the label pass starts one round later)
  const bool tailed = hctl->tail == 2;
  const int rounds_done = tailed ? hctl->tail_round + 1 : hctl->cur;
  const int regular_rounds = tailed ? hctl->tail_round : hctl->cur;
  if (!eager) {  // the kernels the graph ran (the second loop's rounds run the tail's three too)
    const int first_loop = hctl->tail_backs ? hctl->tail_first_back : regular_rounds;
    count_launches(4LL * first_loop + 3 + 7LL * (regular_rounds - first_loop));
  }
  if (labels_out) {
    for (int r = rounds_done - 2; r >= 0; --r) {
      const int64_t Cr = (int64_t)hctl->st[r].C;
      if (Cr == 0) continue;
      const int64_t base = (int64_t)hctl->st[r].pool_at;
      const int64_t nbase = (int64_t)hctl->st[r + 1].pool_at;
      RST_LAUNCH(k_label_back, grid_for(Cr), kBlock, 0, s)(Cr, b.nextpool + base, b.minvpool + base,
                                                          b.minvpool + nbase);
    }
    RST_LAUNCH(k_label_vertices, gN, kBlock, 0, s)(n, b.C1, b.minvpool, labels_out);
    RST_CUDA(cudaGetLastError());
  }
  prof_mark(s, "cc_finish");
  set_stat(STAT_C1, (long long)hctl->st[0].C);
  set_stat(STAT_E2, (long long)hctl->st[1].E);
  out->T = (int64_t)h[CNT_PAIRS];
  out->pairs = b.pairs;
  out->bits = b.bits;
  out->nroots = (int64_t)h[CNT_ROOTS];
  out->roots = b.roots;
  out->rounds = regular_rounds + (tailed ? hctl->tail_rounds : 0) + 1;
  out->root_label = root >= 0 ? hctl->root_label : -1;
  out->rk = pre_rk;
  out->rk_tmp = pre_tmp;
  out->root_bits = pre_root;
  out->rs = pre_rs;
  set_stat(STAT_ROUNDS, out->rounds);
  set_stat(STAT_TAIL, tailed ? hctl->tail_rounds : 0);
  set_stat(STAT_TAIL_BACKS, hctl->tail_backs);
  set_stat(STAT_SPARSE, hctl->giant >= 0 ? (long long)hctl->ng : -1);
  set_stat(STAT_T, out->T);
  set_stat(STAT_NROOTS, out->nroots);
  return RST_OK;
}

// Round 1 alone (the sampled connectivity strategy starts from it): P ends
// as every vertex's round-1 root, pairs[0, counters[0]) holds the tree-edge
// records and bits marks both of their arcs (bits must start zeroed).
template <class OffT>
rst_status round1_forest(const OffT* off, const int32_t* col, int64_t n, int32_t* P, uint32_t* J,
                         uint4* pairs, uint32_t* bits, unsigned long long* counters, cudaStream_t s) {
  uint32_t* status = state().status;
  const int gN = grid_for(n);
  RST_LAUNCH(k_r1_choose<OffT>, gN, kBlock, 0, s)(off, col, n, P, J, nullptr, nullptr, status);
  RST_LAUNCH((k_r1_resolve<OffT, kR1Per, kR1BlocksPerSm>), grid_for((n + kR1Per - 1) / kR1Per, kBlock, kR1BlocksPerSm), kBlock, 0, s)(
      off, col, n, P, J, nullptr, pairs, bits, nullptr, counters, status);
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}
template rst_status round1_forest<int32_t>(const int32_t*, const int32_t*, int64_t, int32_t*, uint32_t*, uint4*,
                                           uint32_t*, unsigned long long*, cudaStream_t);
template rst_status round1_forest<int64_t>(const int64_t*, const int32_t*, int64_t, int32_t*, uint32_t*, uint4*,
                                           uint32_t*, unsigned long long*, cudaStream_t);

template rst_status cc_run<int32_t>(Arena&, const int32_t*, const int32_t*, int64_t, int64_t,
                                    int32_t, int32_t*, CcOut*, cudaStream_t, bool);
template rst_status cc_run<int64_t>(Arena&, const int64_t*, const int32_t*, int64_t, int64_t,
                                    int32_t, int32_t*, CcOut*, cudaStream_t, bool);
template size_t cc_workspace_bytes<int32_t>(int64_t, int64_t);
template size_t cc_workspace_bytes<int64_t>(int64_t, int64_t);

}  // namespace rst
