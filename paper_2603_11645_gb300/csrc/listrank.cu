// Parallel list ranking (Section III-D: every arc gets its position in its
// tree's Euler tour, each tree ranked independently).
//
// Sparse ruling set with recursion.  Every K-th element by index (K = 2^sh,
// 16 unless rst_set_option("lr_spacing") changes it; 8 on the deeper levels)
// and every list head is a splitter; one thread per splitter walks its sublist up to the
// next splitter, reading the successor array (read-only) and writing one
// 8-byte {owner splitter, offset} record per element to a separate array.
// (Overwriting the successor record in place is several times slower on
// GB300: the store to the address just loaded stalls the dependent chain.)
// On the first level the record is packed into 32 bits (owner in the high
// bits, offset in the low ones; an offset that does not fit goes to a full
// 8-byte record): the scattered writes then land in an array half the size,
// which L2 holds far better, and the walk runs about a quarter faster.
// The splitters form a shorter weighted list, ranked the same way until it fits
// one block's shared memory, where Wyllie pointer jumping finishes it.  A
// final coalesced pass adds each owner's position to the element's offset;
// at the first level a caller that only needs some positions can skip it and
// read them from the records (lr_position).
//
// Element indices follow the lexicographic arc order, unrelated to tour
// order, so index-spaced splitters sample the tour uniformly: gaps average K.
// Walks are bounded by N steps; the first level also counts visited elements,
// so an element on a cycle without a head (the input was not a forest) is
// reported instead of silently left unranked.
#include "pipeline.cuh"

namespace rst {

constexpr int kLrMinShift = 4, kLrMaxShift = 9;  // splitter spacing 2^sh: 16 (default) .. 512
constexpr int kLrBase = 4096;            // shared-memory Wyllie base case
constexpr int kLrBaseThreads = 1024;
constexpr int kLrWalkThreads = 128;

constexpr int kLrMaxLevels = 24;  // N < 2^32 shrinks by ~K per level

// Levels after the first use a closer spacing: their lists are short and
// L2-resident, so a level's time is its longest sublist (about K ln S steps
// of dependent L2 reads), not its bytes.
constexpr int kLrDeepShift = 3;
static int level_shift(int level, int sh) { return level == 0 || sh < kLrDeepShift ? sh : kLrDeepShift; }

struct LevelBufs {
  int2* ol;         // N {owner, offset} records of this level
  uint32_t* ol32;   // level 0: the same packed into 32 bits (null: unpacked)
  int32_t* snext;   // S successors of the next level
  uint32_t* w_next; // S weights of the next level
  int32_t* sstart;  // S (only the head slots are used)
  int32_t* shead;   // h
  uint32_t* spos;   // S positions of the splitters
};

static int64_t lr_splitters(int64_t N, int64_t h, int sh) { return ((N + (1LL << sh) - 1) >> sh) + h; }

// Walks the workspace plan: identical calls for the counting pass and the run.
// Fixed-capacity level list (no host allocation on the ranking path).
struct LevelList {
  LevelBufs b[kLrMaxLevels];
  int count = 0;
  void push_back(const LevelBufs& x) {
    if (count < kLrMaxLevels) b[count] = x;
    ++count;
  }
};

static void lr_layout(Arena& ar, int64_t N, int64_t h, int sh, LevelList* levels,
                      int32_t** wyl_pj, uint32_t** wyl_val, int32_t** wyl_flag) {
  bool first = true;
  for (int l = 0; N > kLrBase && h <= N / 4; ++l) {
    const int64_t S = lr_splitters(N, h, level_shift(l, sh));
    LevelBufs b;
    b.ol = ar.take<int2>(N);
    b.ol32 = first ? ar.take<uint32_t>(N) : nullptr;
    first = false;
    b.snext = ar.take<int32_t>(S);
    b.w_next = ar.take<uint32_t>(S);
    b.sstart = ar.take<int32_t>(S);
    b.shead = ar.take<int32_t>(h);
    b.spos = ar.take<uint32_t>(S);
    if (levels) levels->push_back(b);
    N = S;
  }
  if (N > kLrBase) {  // many short lists: global Wyllie
    *wyl_pj = ar.take<int32_t>(2 * N);
    *wyl_val = ar.take<uint32_t>(2 * N);
    *wyl_flag = ar.take<int32_t>(1);
  }
}

// Bytes for any allowed spacing (the largest of the layouts), so the spacing
// can change between calls without resizing.
size_t list_rank_workspace_bytes(int64_t N, int64_t nheads) {
  size_t most = 0;
  for (int sh = kLrMinShift; sh <= kLrMaxShift; ++sh) {
    Arena a;
    a.counting = true;
    int32_t* p = nullptr;
    uint32_t* v = nullptr;
    int32_t* f = nullptr;
    lr_layout(a, N, nheads, sh, nullptr, &p, &v, &f);
    if (a.used > most) most = a.used;
  }
  return most;
}

size_t list_rank_workspace_upper(int64_t N) {
  size_t best = 0;
  const int64_t hs[] = {1, N / 256, N / 64, N / 16, N / 5, N / 4 + 1, N / 2 + 1, N};
  for (int64_t h : hs) {
    size_t b = list_rank_workspace_bytes(N, h < 1 ? 1 : h);
    if (b > best) best = b;
  }
  return best;
}

__device__ __forceinline__ uint32_t wget(const uint32_t* w, int64_t x) { return w ? w[x] : 1u; }

__global__ void k_lr_heads(int64_t N, int64_t S0, int sh, const int32_t* __restrict__ heads, int64_t h,
                           int32_t* __restrict__ sstart, int32_t* __restrict__ shead) {
  pdl_wait();  // launched as a programmatic dependent
  const int32_t mask = (1 << sh) - 1;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < h;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = heads[j];
    if (x < 0) {  // a list without elements: no splitter
      shead[j] = -1;
      sstart[S0 + j] = -1;
    } else if ((x & mask) == 0) {
      shead[j] = x >> sh;
      sstart[S0 + j] = -1;
    } else {
      shead[j] = (int32_t)(S0 + j);
      sstart[S0 + j] = x;
    }
  }
}

// One thread per splitter: ol[x] = {owner splitter, weighted offset}.
__global__ void __launch_bounds__(kLrWalkThreads) k_lr_walk(int64_t N, int64_t S0, int64_t S, int sh,
                                                            const int32_t* __restrict__ nxt,
                                                            const uint32_t* __restrict__ w,
                                                            const int32_t* __restrict__ sstart,
                                                            int2* __restrict__ ol,
                                                            uint32_t* __restrict__ ol32, int fbits,
                                                            int32_t* __restrict__ snext,
                                                            uint32_t* __restrict__ w_next,
                                                            unsigned long long* visited,
                                                            uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  unsigned long long seen = 0;
  const int32_t mask = (1 << sh) - 1;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t start = s < S0 ? s << sh : (int64_t)sstart[s];
    if (start < 0) {
      snext[s] = -1;
      w_next[s] = 0;
      continue;
    }
    // packed records (first level, unit weights): owner in the high bits,
    // offset in the low fbits; an offset that does not fit is written to ol
    // and marked by the all-ones word
    const uint32_t omax = ol32 ? (1u << fbits) - 1u : 0u;
    const uint32_t ohi = ol32 ? (uint32_t)s << fbits : 0u;
    if (ol32)
      ol32[start] = ohi;
    else
      ol[start] = make_int2((int32_t)s, 0);
    uint32_t acc = wget(w, start);
    int32_t x = nxt[start];
    int64_t steps = 1;
    while (x >= 0 && (x & mask) != 0) {
      if (ol32) {
        if (acc < omax) {
          ol32[x] = ohi | acc;
        } else {
          ol32[x] = 0xffffffffu;
          ol[x] = make_int2((int32_t)s, (int32_t)acc);
        }
      } else {
        ol[x] = make_int2((int32_t)s, (int32_t)acc);
      }
      acc += wget(w, x);
      x = nxt[x];
      if (++steps > N) {
        raise_error(status, DERR_WALK_LIMIT);
        x = -1;
        break;
      }
    }
    snext[s] = x < 0 ? -1 : x >> sh;
    w_next[s] = acc;
    seen += (unsigned long long)steps;
  }
  if (visited) {
    for (int d = 16; d > 0; d >>= 1) seen += __shfl_down_sync(0xffffffffu, seen, d);
    if ((threadIdx.x & 31) == 0 && seen) atomicAdd(visited, seen);
  }
}

// pos[x] = position of x's owner + x's offset.  At the first level every
// element must have been visited (visited == N); at deeper levels the unused
// slots of heads that coincided with a regular splitter are never visited.
// An unvisited element's record holds whatever the workspace held before, so
// the owner index is bounds-checked (S = number of splitters) before use.
__global__ void k_lr_final(int64_t N, int64_t S, const int2* __restrict__ ol,
                           const uint32_t* __restrict__ ol32, int fbits,
                           const uint32_t* __restrict__ spos, uint32_t* __restrict__ pos,
                           const unsigned long long* visited, uint32_t* status) {
  pdl_wait();  // launched as a programmatic dependent
  if (visited && blockIdx.x == 0 && threadIdx.x == 0 && *visited != (unsigned long long)N)
    raise_error(status, DERR_NOT_FOREST);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x)
    pos[x] = lr_position(ol, ol32, fbits, spos, S, (uint32_t)x);
}

// Base case in one block: predecessor pointers, then Wyllie pointer jumping
// with a read phase and a write phase per round.
__global__ void __launch_bounds__(kLrBaseThreads) k_lr_base(int64_t N, const int32_t* __restrict__ nxt,
                                                            const uint32_t* __restrict__ w,
                                                            uint32_t* __restrict__ pos) {
  pdl_wait();  // launched as a programmatic dependent
  __shared__ int32_t pj[kLrBase];
  __shared__ uint32_t val[kLrBase];
  const int n = (int)N;
  for (int x = threadIdx.x; x < n; x += blockDim.x) pj[x] = -1;
  __syncthreads();
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    const int32_t y = nxt[x];
    if (y >= 0 && y < n) pj[y] = x;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n; x += blockDim.x) val[x] = pj[x] >= 0 ? wget(w, pj[x]) : 0u;
  __syncthreads();
  constexpr int kPer = kLrBase / kLrBaseThreads;
  for (int round = 0; (1 << round) < n + 1; ++round) {
    int32_t np[kPer];
    uint32_t nv[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int x = threadIdx.x + k * kLrBaseThreads;
      if (x < n) {
        const int32_t p = pj[x];
        np[k] = p >= 0 ? pj[p] : -1;
        nv[k] = p >= 0 ? val[x] + val[p] : val[x];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int x = threadIdx.x + k * kLrBaseThreads;
      if (x < n) {
        pj[x] = np[k];
        val[x] = nv[k];
      }
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < n; x += blockDim.x) pos[x] = val[x];
}

// Global-memory Wyllie for levels with many short lists.
__global__ void k_wyl_init(int64_t N, const int32_t* __restrict__ nxt, const uint32_t* __restrict__ w,
                           int32_t* __restrict__ pj, uint32_t* __restrict__ val) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t y = nxt[x];
    if (y >= 0 && y < N) {
      pj[y] = (int32_t)x;
      val[y] = wget(w, x);
    }
  }
}

__global__ void k_wyl_round(int64_t N, const int32_t* __restrict__ pj, const uint32_t* __restrict__ val,
                            int32_t* __restrict__ pj2, uint32_t* __restrict__ val2, int32_t* flag) {
  bool any = false;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pj[x];
    if (p >= 0) {
      pj2[x] = pj[p];
      val2[x] = val[x] + val[p];
      any = any || pj[p] >= 0;
    } else {
      pj2[x] = -1;
      val2[x] = val[x];
    }
  }
  if (any) *flag = 1;
}

rst_status list_rank(Arena& ar, int64_t N, const int32_t* nxt, const uint32_t* w, const int32_t* heads,
                     int64_t nheads, uint32_t* pos, cudaStream_t s, LrFirstLevel* first) {
  if (first) first->valid = false;
  if (N <= 0) return RST_OK;
  LevelList levels;
  int32_t* wpj = nullptr;
  uint32_t* wval = nullptr;
  int32_t* wflag = nullptr;
  const int sh = tuning().lr_shift;
  lr_layout(ar, N, nheads, sh, &levels, &wpj, &wval, &wflag);
  if (levels.count > kLrMaxLevels) return RST_ERR_UNSUPPORTED;
  if (ar.used > ar.cap) return RST_ERR_OOM;  // some buffer of the layout did not fit (null)
  set_stat(STAT_LEVELS, (long long)levels.count);
  set_stat(STAT_LR_N, N);
  uint32_t* status = state().status;
  unsigned long long* visited = dev_counter(7);

  struct Frame {
    int64_t N;
    const int32_t* nxt;
    const uint32_t* w;
    const int32_t* heads;
    uint32_t* pos;
  };
  Frame frames[kLrMaxLevels];
  int lfbits[kLrMaxLevels] = {};
  Frame f{N, nxt, w, heads, pos};
  for (int l = 0; l < levels.count; ++l) {
    LevelBufs& b = levels.b[l];
    const int shl = level_shift(l, sh);
    const int64_t S0 = (f.N + (1LL << shl) - 1) >> shl;
    const int64_t S = S0 + nheads;
    if (l == 0) RST_CUDA(cudaMemsetAsync(visited, 0, sizeof(unsigned long long), s));
    RST_LAUNCH_PDL(k_lr_heads, grid_for(nheads), kBlock, 0, s)(f.N, S0, shl, f.heads, nheads, b.sstart, b.shead);
    prof_mark(s, l == 0 ? "lr_prep1" : "lr_prep");
    int obits = 1;
    while (((int64_t)1 << obits) < S) ++obits;
    const int fbits = 32 - obits;
    if (fbits < 8) b.ol32 = nullptr;  // too many splitters to pack: full records
    lfbits[l] = fbits;
    RST_LAUNCH_PDL(k_lr_walk, (unsigned)((S + kLrWalkThreads - 1) / kLrWalkThreads), kLrWalkThreads, 0, s)(
        f.N, S0, S, shl, f.nxt, f.w, b.sstart, b.ol, b.ol32, fbits, b.snext, b.w_next,
        l == 0 ? visited : nullptr, status);
    prof_mark(s, l == 0 ? "k_lr_walk1" : "k_lr_walk");
    RST_CUDA(cudaGetLastError());
    frames[l] = f;
    f = Frame{S, b.snext, b.w_next, b.shead, b.spos};
  }
  if (f.N <= kLrBase) {
    RST_LAUNCH_PDL(k_lr_base, 1, kLrBaseThreads, 0, s)(f.N, f.nxt, f.w, f.pos);
  } else {
    RST_CUDA(cudaMemsetAsync(wpj, 0xff, f.N * sizeof(int32_t), s));
    RST_CUDA(cudaMemsetAsync(wval, 0, f.N * sizeof(uint32_t), s));
    RST_LAUNCH(k_wyl_init, grid_for(f.N), kBlock, 0, s)(f.N, f.nxt, f.w, wpj, wval);
    int32_t* pa = wpj;
    int32_t* pb = wpj + f.N;
    uint32_t* va = wval;
    uint32_t* vb = wval + f.N;
    for (int round = 0; round < 40; ++round) {
      RST_CUDA(cudaMemsetAsync(wflag, 0, sizeof(int32_t), s));
      RST_LAUNCH(k_wyl_round, grid_for(f.N), kBlock, 0, s)(f.N, pa, va, pb, vb, wflag);
      std::swap(pa, pb);
      std::swap(va, vb);
      int32_t hf = 0;
      RST_CUDA(cudaMemcpyAsync(state().hostbuf, wflag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RST_CUDA(cudaStreamSynchronize(s));
      std::memcpy(&hf, state().hostbuf, sizeof(int32_t));
      if (!hf) break;
      if (round == 39) return RST_ERR_NOT_CONVERGED;
    }
    RST_CUDA(cudaMemcpyAsync(f.pos, va, f.N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  prof_mark(s, "lr_base");
  RST_CUDA(cudaGetLastError());
  for (int l = levels.count - 1; l >= 0; --l) {
    const Frame& fr = frames[l];
    LevelBufs& b = levels.b[l];
    const int shl = level_shift(l, sh);
    const int64_t S = ((fr.N + (1LL << shl) - 1) >> shl) + nheads;
    if (l == 0 && first) {  // the caller reads positions from the records
      first->valid = true;
      first->ol = b.ol;
      first->ol32 = b.ol32;
      first->fbits = lfbits[0];
      first->spos = b.spos;
      first->S = S;
      first->visited = visited;
      first->N = fr.N;
      break;
    }

    RST_LAUNCH_PDL(k_lr_final, grid_for(fr.N), kBlock, 0, s)(fr.N, S, b.ol, b.ol32, lfbits[l], b.spos, fr.pos,
                                                         l == 0 ? visited : nullptr, status);
    prof_mark(s, l == 0 ? "k_lr_final1" : "k_lr_final");
  }
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}

}  // namespace rst
