// Shared device/host utilities of the RST library (not part of the C ABI).
#pragma once
#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <cstring>
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "rst.h"

namespace rst {

// ------------------------------------------------------------------ errors
// Device-detected error bits, OR-ed into the per-device status word.
enum DeviceError : uint32_t {
  DERR_INDEX = 1u << 0,        // an index read from input memory was out of range
  DERR_WALK_LIMIT = 1u << 1,   // a list walk exceeded its iteration bound
  DERR_NOT_FOREST = 1u << 2,   // Euler input was not a forest
  DERR_ROUND_LIMIT = 1u << 3,  // an iterative phase exceeded its round bound
  DERR_CAPACITY = 1u << 4,     // an internal list overflowed its planned size
};

#define RST_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) {                              \
      ::rst::note_cuda_error(e__, #call, __FILE__, __LINE__); \
      return RST_ERR_CUDA;                                 \
    }                                                      \
  } while (0)

#define RST_TRY(expr)                     \
  do {                                    \
    rst_status s__ = (expr);              \
    if (s__ != RST_OK) return s__;        \
  } while (0)

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// ------------------------------------------------------------------ instrumentation
// Every kernel launch goes through RST_LAUNCH so that the library can report
// how many of its kernels ran (rst_launch_count).
void count_launch();
void count_launches(long long k);  // kernels executed inside a graph launch
#define RST_LAUNCH(k, ...) ::rst::count_launch(), k<<<__VA_ARGS__>>>

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel on the stream drains (its launch latency and first blocks
// overlap that kernel's tail).  Every kernel launched this way calls
// pdl_wait() before it touches memory, which waits until the previous grid
// has completed and its writes are visible; in a kernel launched plainly
// pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <class... P>
struct PdlLaunch {
  void (*f)(P...);
  dim3 grid, block;
  size_t smem;
  cudaStream_t stream;
  template <class... A>
  void operator()(A&&... a) const {
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, f, std::forward<A>(a)...);  // errors surface through cudaGetLastError
  }
};
template <class... P>
inline PdlLaunch<P...> pdl_launch(void (*f)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
  return PdlLaunch<P...>{f, grid, block, smem, s};
}
// RST_LAUNCH_PDL(kernel, grid, block, smem, stream)(args...); a templated
// kernel name goes in parentheses.
#define RST_LAUNCH_PDL(...) ::rst::pdl_launch(__VA_ARGS__)
// Stage marks: when profiling is on, records a CUDA event on `s` that ends the
// stage `name` (a string literal); rst_profile_read returns the durations.
void prof_mark(cudaStream_t s, const char* name);
// Sizes seen by the last call (read through rst_last_stats).
enum StatSlot : int {
  STAT_ROUNDS = 0,   // hooking rounds
  STAT_C1 = 1,       // components after round 1 that still have edges
  STAT_E2 = 2,       // inter-component edges after round 1
  STAT_T = 3,        // tree edges
  STAT_NROOTS = 4,   // components with edges
  STAT_LEVELS = 5,   // BFS levels (BFS) / list-ranking levels (CC+Euler)
  STAT_LR_N = 6,     // elements list-ranked (tree arcs left after leaf pruning)
  STAT_TAIL = 7,     // CC+Euler: rounds the single-block tail ran (0: it did not finish the rounds)
  STAT_TAIL_BACKS = 8,  // CC+Euler: times the tail's component pairs did not fit
  STAT_SPARSE = 9,   // CC+Euler: rows the list build read outside a giant round-1 component (-1: all rows)
  STAT_COUNT = 10
};
void set_stat(int slot, long long v);

// ------------------------------------------------------------------ launch
constexpr int kBlock = 256;

struct Device {
  int id = -1;
  int sms = 152;
  int max_threads_per_sm = 2048;
};
const Device& device_info();

// Launch and sampling parameters that change no result, only speed; set by
// rst_set_option (an offline tuner picks them per size bucket).  Process-wide:
// change them only between calls.
struct Tuning {
  int lr_shift = 4;     // list ranking: one splitter per 2^lr_shift elements (16..512)
  int round_bps = 8;    // contraction-round kernels: resident blocks per SM in the grid (1..16)
  int bfs_bu_div = 20;  // BFS steps bottom-up while the frontier exceeds n / bfs_bu_div
  int bfsd_bps = 2;     // device-driven BFS: 256-thread blocks per SM in its grid (1..8)
  int bfsp_bps = 1;     // persistent BFS: at most this many resident blocks per SM (1..8)
  long long insert_walk_limit = 2048;  // edge insertion: sparse rounds while walks to roots stay this short (0: never)
  int euler_block = 256;  // block size of the tour's grid-stride kernels (run flags, successors, parents): 128/256/512
  int pr_levels = 1;      // PR-RST: pointer-jumping levels computed per launch and host check (1..3)
  int giant_pct = 75;     // list build from the rows outside a round-1 component holding this
                          // percentage of the sampled vertices (0: the largest always; 101: never)
};
Tuning& tuning();

// Grid for a grid-stride loop over `work` items: at most `waves` resident
// blocks per SM, at least 1 block.
inline int grid_for(int64_t work, int block = kBlock, int waves = 8) {
  const Device& d = device_info();
  int64_t need = (work + block - 1) / block;
  int64_t cap = (int64_t)d.sms * waves;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

// ------------------------------------------------------------------ workspace
// Bump allocator over one grow-only device buffer per device.  A call first
// plans its buffers with a counting pass (base == nullptr), ensures capacity,
// then takes them for real.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool counting = false;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    size_t at = used;
    used += bytes;
    if (counting) return nullptr;
    if (used > cap) return nullptr;
    return reinterpret_cast<T*>(base + at);
  }
};

struct DeviceState {
  char* ws = nullptr;          // workspace
  size_t ws_cap = 0;
  uint32_t* status = nullptr;  // device error word + small scalars (64 words)
  unsigned long long* hostbuf = nullptr;  // pinned host scratch (kHostBufWords words)
  cudaEvent_t readback = nullptr;         // marks a read-back inside a longer stream (may be null)
};
constexpr int kHostBufWords = 512;

// Per-device state and the process-wide call lock.  A call that must not
// allocate installs its own DeviceState (fixed buffers) for the current host
// thread with set_state_override; state() then returns it.
DeviceState& state();
void set_state_override(DeviceState* st);
bool state_overridden();
// Host scratch for small device->host reads (static storage, calls are serialised).
void* host_scratch(size_t bytes);
std::mutex& call_lock();
rst_status ensure_workspace(size_t bytes);

// Small device scalars live in state().status[...]
enum ScalarSlot : int {
  SLOT_ERR = 0,
  SLOT_COUNT0 = 8,   // 64-bit counters at even slots 8.. (unsigned long long view)
};

inline unsigned long long* dev_counter(int k) {
  return reinterpret_cast<unsigned long long*>(state().status + 8) + k;
}

rst_status read_device_error(cudaStream_t s);
rst_status reset_device_error(cudaStream_t s);
// Copy `count` 64-bit words from device to the pinned host buffer and wait.
rst_status fetch_u64(const unsigned long long* dsrc, int count, unsigned long long* out,
                     cudaStream_t s);

__device__ __forceinline__ void raise_error(uint32_t* status, uint32_t bits) {
  atomicOr(status, bits);
}

// ------------------------------------------------------------------ warp helpers
// Warp-aggregated reservation of slots in an append buffer.  Every lane of the
// warp must call it (pred may differ).  Returns the slot or -1.
__device__ __forceinline__ long long warp_reserve(unsigned long long* counter, bool pred) {
  const unsigned full = 0xffffffffu;
  unsigned m = __ballot_sync(full, pred);
  int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (m != 0) {
    int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(full, base, leader);
  }
  return pred ? (long long)(base + __popc(m & ((1u << lane) - 1u))) : -1;
}

// Block-aggregated reservation: every thread of the block calls it (with its
// own count, possibly 0); one atomicAdd per block.  Returns the first slot of
// this thread's range.  Contains __syncthreads(): call from block-uniform code.
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_reserve(unsigned long long* counter,
                                                           unsigned int cnt) {
  constexpr int kWarps = BLOCK / 32;
  __shared__ unsigned int s_warp[kWarps];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int x = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const unsigned int w = lane < kWarps ? s_warp[lane] : 0u;
    unsigned int ws = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, ws, d);
      if (lane >= d) ws += y;
    }
    if (lane < kWarps) s_warp[lane] = ws - w;
    if (lane == kWarps - 1) s_base = ws ? atomicAdd(counter, (unsigned long long)ws) : 0ull;
  }
  __syncthreads();
  const unsigned long long r = s_base + s_warp[warp] + (x - cnt);
  __syncthreads();
  return r;
}

// Streams read or written once, marked evict-first in L2 (createpolicy +
// .L2::cache_hint), so that they do not push out the arrays the same kernel
// gathers from or scatters into.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_stream(uint4* p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sums over 64-bit values: out[i] = sum(in[0..i)), and
// out[count] = total.  `in` may alias `out`.  tmp needs scan_tmp_words(count).
size_t scan_tmp_words(int64_t count);
rst_status scan_exclusive_u64(const unsigned long long* in, unsigned long long* out,
                              int64_t count, unsigned long long* tmp, cudaStream_t s);
// Same over 32-bit words of a bitmap: out[w] = popcount of words [0, w).
rst_status scan_popcount_words(const uint32_t* words, uint32_t* out, int64_t count,
                               unsigned long long* tmp, cudaStream_t s);
// The same interleaved with the words: out[i] = {words[i], popcount of words
// [0, i)} for i < count, out[count] = {0, total}.
rst_status scan_popcount_ranked(const uint32_t* words, uint2* out, int64_t count,
                                unsigned long long* tmp, cudaStream_t s);

}  // namespace rst
