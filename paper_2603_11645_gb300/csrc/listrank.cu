// Parallel list ranking (Section III-D: "parallel list ranking assigns each
// edge its position within its respective Euler tour").
//
// Sparse ruling set with recursion: every K-th element (by index) and every
// list head is a splitter; one thread per splitter walks its sublist up to
// the next splitter, recording (owner splitter, offset) for each element and
// the weighted gap to the next splitter.  The splitters form a shorter
// weighted list that is ranked the same way until it fits one block's shared
// memory, where Wyllie pointer jumping finishes it.  A final pass adds the
// splitter's position to each element's offset.
//
// Indices of the successor array follow the lexicographic arc order, which is
// unrelated to tour order, so the index-spaced splitters are a uniform random
// sample of the tour: gaps average K.  Every walk is bounded by N steps; a
// longer walk (a cycle without a head: the input was not a forest) sets an
// error bit and stops.
#include "pipeline.cuh"

namespace rst {

constexpr int kLrK = 16;                 // splitter spacing (power of two)
constexpr int kLrBase = 4096;            // shared-memory Wyllie base case
constexpr int kLrBaseThreads = 1024;

struct LevelBufs {
  int32_t* owner;   // N
  uint32_t* local;  // N
  int32_t* snext;   // S
  uint32_t* slen;   // S
  int32_t* sstart;  // S
  int32_t* shead;   // h
  uint32_t* spos;   // S
};

static int64_t lr_splitters(int64_t N, int64_t h) { return (N + kLrK - 1) / kLrK + h; }

// Walks the workspace plan: identical calls for the counting pass and the run.
static void lr_layout(Arena& ar, int64_t N, int64_t h, std::vector<LevelBufs>* levels,
                      int32_t** wyl_pj, uint32_t** wyl_val, int32_t** wyl_flag) {
  while (N > kLrBase && h <= N / 4) {
    const int64_t S = lr_splitters(N, h);
    LevelBufs b;
    b.owner = ar.take<int32_t>(N);
    b.local = ar.take<uint32_t>(N);
    b.snext = ar.take<int32_t>(S);
    b.slen = ar.take<uint32_t>(S);
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

size_t list_rank_workspace_bytes(int64_t N, int64_t nheads) {
  Arena a;
  a.counting = true;
  int32_t* p = nullptr;
  uint32_t* v = nullptr;
  int32_t* f = nullptr;
  lr_layout(a, N, nheads, nullptr, &p, &v, &f);
  return a.used;
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

__global__ void k_lr_heads(int64_t N, int64_t S0, const int32_t* __restrict__ heads, int64_t h,
                           int32_t* __restrict__ sstart, int32_t* __restrict__ shead) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < h;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = heads[j];
    if ((x & (kLrK - 1)) == 0) {
      shead[j] = x / kLrK;
      sstart[S0 + j] = -1;
    } else {
      shead[j] = (int32_t)(S0 + j);
      sstart[S0 + j] = x;
    }
  }
}

__global__ void k_lr_walk(int64_t N, int64_t S0, int64_t S, const int32_t* __restrict__ nxt,
                          const uint32_t* __restrict__ w, const int32_t* __restrict__ sstart,
                          int32_t* __restrict__ owner, uint32_t* __restrict__ local,
                          int32_t* __restrict__ snext, uint32_t* __restrict__ slen,
                          uint32_t* status) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t start = s < S0 ? s * kLrK : (int64_t)sstart[s];
    if (start < 0) {
      snext[s] = -1;
      slen[s] = 0;
      continue;
    }
    owner[start] = (int32_t)s;
    local[start] = 0;
    uint32_t acc = wget(w, start);
    int32_t x = nxt[start];
    int64_t steps = 0;
    while (x >= 0 && (x & (kLrK - 1)) != 0) {
      owner[x] = (int32_t)s;
      local[x] = acc;
      acc += wget(w, x);
      x = nxt[x];
      if (++steps > N) {
        raise_error(status, DERR_WALK_LIMIT);
        x = -1;
        break;
      }
    }
    snext[s] = x < 0 ? -1 : x / kLrK;
    slen[s] = acc;
  }
}

// Elements no walk reached: at the first level they lie on a cycle without a
// head (the input was not a forest); at deeper levels they are the unused
// slots of heads that coincided with a regular splitter, and are ignored.
__global__ void k_lr_final(int64_t N, const int32_t* __restrict__ owner,
                           const uint32_t* __restrict__ local, const uint32_t* __restrict__ spos,
                           uint32_t* __restrict__ pos, int first_level, uint32_t* status) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = owner[x];
    if (o < 0) {
      if (first_level) raise_error(status, DERR_NOT_FOREST);
      pos[x] = kNone;
    } else {
      pos[x] = spos[o] + local[x];
    }
  }
}

// Base case in one block: predecessor pointers, then Wyllie pointer jumping
// with a read phase and a write phase per round.
__global__ void __launch_bounds__(kLrBaseThreads) k_lr_base(int64_t N, const int32_t* __restrict__ nxt,
                                                            const uint32_t* __restrict__ w,
                                                            uint32_t* __restrict__ pos) {
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

rst_status list_rank(Arena& ar, int64_t N, const int32_t* nxt, const uint32_t* w,
                     const int32_t* heads, int64_t nheads, uint32_t* pos, cudaStream_t s) {
  if (N <= 0) return RST_OK;
  std::vector<LevelBufs> levels;
  int32_t* wpj = nullptr;
  uint32_t* wval = nullptr;
  int32_t* wflag = nullptr;
  lr_layout(ar, N, nheads, &levels, &wpj, &wval, &wflag);
  for (auto& b : levels)
    if (!b.spos) return RST_ERR_OOM;
  uint32_t* status = state().status;

  // descend
  struct Frame {
    int64_t N;
    const int32_t* nxt;
    const uint32_t* w;
    const int32_t* heads;
    uint32_t* pos;
  };
  std::vector<Frame> frames;
  Frame f{N, nxt, w, heads, pos};
  for (size_t l = 0; l < levels.size(); ++l) {
    LevelBufs& b = levels[l];
    const int64_t S0 = (f.N + kLrK - 1) / kLrK;
    const int64_t S = S0 + nheads;
    RST_CUDA(cudaMemsetAsync(b.owner, 0xff, f.N * sizeof(int32_t), s));
    k_lr_heads<<<grid_for(nheads), kBlock, 0, s>>>(f.N, S0, f.heads, nheads, b.sstart, b.shead);
    k_lr_walk<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(f.N, S0, S, f.nxt, f.w, b.sstart, b.owner,
                                                    b.local, b.snext, b.slen, status);
    RST_CUDA(cudaGetLastError());
    frames.push_back(f);
    f = Frame{S, b.snext, b.slen, b.shead, b.spos};
  }
  // base
  if (f.N <= kLrBase) {
    k_lr_base<<<1, kLrBaseThreads, 0, s>>>(f.N, f.nxt, f.w, f.pos);
  } else {
    RST_CUDA(cudaMemsetAsync(wpj, 0xff, f.N * sizeof(int32_t), s));
    RST_CUDA(cudaMemsetAsync(wval, 0, f.N * sizeof(uint32_t), s));
    k_wyl_init<<<grid_for(f.N), kBlock, 0, s>>>(f.N, f.nxt, f.w, wpj, wval);
    int32_t* pa = wpj;
    int32_t* pb = wpj + f.N;
    uint32_t* va = wval;
    uint32_t* vb = wval + f.N;
    for (int round = 0; round < 40; ++round) {
      RST_CUDA(cudaMemsetAsync(wflag, 0, sizeof(int32_t), s));
      k_wyl_round<<<grid_for(f.N), kBlock, 0, s>>>(f.N, pa, va, pb, vb, wflag);
      std::swap(pa, pb);
      std::swap(va, vb);
      int32_t hf = 0;
      RST_CUDA(cudaMemcpyAsync(&hf, wflag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RST_CUDA(cudaStreamSynchronize(s));
      if (!hf) break;
      if (round == 39) return RST_ERR_NOT_CONVERGED;
    }
    RST_CUDA(cudaMemcpyAsync(f.pos, va, f.N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  RST_CUDA(cudaGetLastError());
  // ascend
  for (int l = (int)levels.size() - 1; l >= 0; --l) {
    const Frame& fr = frames[l];
    LevelBufs& b = levels[l];
    k_lr_final<<<grid_for(fr.N), kBlock, 0, s>>>(fr.N, b.owner, b.local, b.spos, fr.pos, l == 0,
                                                  status);
  }
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}

}  // namespace rst
