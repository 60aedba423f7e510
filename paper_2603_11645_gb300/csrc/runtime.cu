// Runtime support: per-device workspace, status word, error reporting, scans.
#include <atomic>
#include <cstring>

#include "common.cuh"
#include <string>

namespace rst {

static thread_local char g_last_error[256] = {0};

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s at %s:%d: %s", cudaGetErrorString(e), file,
           line, what);
  if (getenv("RST_DEBUG")) fprintf(stderr, "[rst] %s\n", g_last_error);
}

static thread_local DeviceState* g_state_override = nullptr;
void set_state_override(DeviceState* st) { g_state_override = st; }
bool state_overridden() { return g_state_override != nullptr; }

alignas(64) static unsigned char g_host_scratch[1 << 16];
void* host_scratch(size_t bytes) { return bytes <= sizeof(g_host_scratch) ? g_host_scratch : nullptr; }

static std::atomic<long long> g_launches{0};
static long long g_stats[STAT_COUNT] = {0};
void set_stat(int slot, long long v) {
  if (slot >= 0 && slot < STAT_COUNT) g_stats[slot] = v;
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct Profiler {
  bool on = false;
  std::vector<std::pair<const char*, cudaEvent_t>> marks;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> only;  // record only these marks (empty: all)
};
static Profiler g_prof;

void prof_mark(cudaStream_t s, const char* name) {
  if (!g_prof.on || g_state_override) return;  // event creation may allocate
  if (!g_prof.only.empty() &&
      std::find(g_prof.only.begin(), g_prof.only.end(), name) == g_prof.only.end())
    return;
  cudaEvent_t e;
  if (g_prof.pool.empty()) {
    if (cudaEventCreate(&e) != cudaSuccess) return;
  } else {
    e = g_prof.pool.back();
    g_prof.pool.pop_back();
  }
  cudaEventRecord(e, s);
  g_prof.marks.emplace_back(name, e);
}

constexpr int kMaxDevices = 64;
static Device g_dev[kMaxDevices];
static DeviceState g_state[kMaxDevices];

static int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) d = 0;
  return d < kMaxDevices ? d : 0;
}

Tuning& tuning() {
  static Tuning t;
  return t;
}

const Device& device_info() {
  int d = current_device();
  Device& info = g_dev[d];
  if (info.id != d) {
    int sms = 0, mt = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    cudaDeviceGetAttribute(&mt, cudaDevAttrMaxThreadsPerMultiProcessor, d);
    info.sms = sms > 0 ? sms : 152;
    info.max_threads_per_sm = mt > 0 ? mt : 2048;
    info.id = d;
  }
  return info;
}


DeviceState& state() { return g_state_override ? *g_state_override : g_state[current_device()]; }

std::mutex& call_lock() {
  static std::mutex m;
  return m;
}

static rst_status ensure_small(DeviceState& st) {
  if (!st.status) {
    RST_CUDA(cudaMalloc(&st.status, 64 * sizeof(uint32_t)));
    RST_CUDA(cudaMemset(st.status, 0, 64 * sizeof(uint32_t)));
  }
  if (!st.hostbuf) {
    RST_CUDA(cudaMallocHost(&st.hostbuf, kHostBufWords * sizeof(unsigned long long)));
  }
  // the read-back event only serves calls with their own workspace; a call
  // running on fixed buffers (state override) creates nothing
  if (!st.readback && !state_overridden()) {
    RST_CUDA(cudaEventCreateWithFlags(&st.readback, cudaEventDisableTiming));
  }
  return RST_OK;
}

rst_status ensure_workspace(size_t bytes) {
  DeviceState& st = state();
  RST_TRY(ensure_small(st));
  if (bytes <= st.ws_cap) return RST_OK;
  if (st.ws) {
    RST_CUDA(cudaDeviceSynchronize());
    RST_CUDA(cudaFree(st.ws));
    st.ws = nullptr;
    st.ws_cap = 0;
  }
  size_t want = bytes + bytes / 8 + (1u << 20);
  cudaError_t e = cudaMalloc(&st.ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    st.ws = nullptr;
    e = cudaMalloc(&st.ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st.ws = nullptr;
      return RST_ERR_OOM;
    }
    want = bytes;
  }
  st.ws_cap = want;
  return RST_OK;
}

rst_status reset_device_error(cudaStream_t s) {
  DeviceState& st = state();
  RST_TRY(ensure_small(st));
  RST_CUDA(cudaMemsetAsync(st.status, 0, 64 * sizeof(uint32_t), s));
  return RST_OK;
}

rst_status fetch_u64(const unsigned long long* dsrc, int count, unsigned long long* out,
                     cudaStream_t s) {
  DeviceState& st = state();
  RST_CUDA(cudaMemcpyAsync(st.hostbuf, dsrc, count * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) out[i] = st.hostbuf[i];
  return RST_OK;
}

rst_status read_device_error(cudaStream_t s) {
  DeviceState& st = state();
  uint32_t err = 0;
  RST_CUDA(cudaMemcpyAsync(st.hostbuf, st.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaStreamSynchronize(s));
  std::memcpy(&err, st.hostbuf, sizeof(uint32_t));
  if (err & (DERR_WALK_LIMIT | DERR_ROUND_LIMIT)) return RST_ERR_NOT_CONVERGED;
  if (err) return RST_ERR_DEVICE;
  return RST_OK;
}

// ------------------------------------------------------------------ scans
// Reduce-then-scan over tiles of kScanTile items: block sums, a single-block
// scan of the sums, then a downsweep that rescans each tile with its offset.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(int64_t count) { return (size_t)((count + kScanTile - 1) / kScanTile) + 2; }

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem_warp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (blockDim.x >> 5) ? smem_warp[lane] : T(0);
    T ws = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, ws, d);
      if (lane >= d) ws += y;
    }
    if (lane < (blockDim.x >> 5)) smem_warp[lane] = ws - w;
    if (lane == (blockDim.x >> 5) - 1) smem_warp[32] = ws;
  }
  __syncthreads();
  T res = x - v + smem_warp[warp];
  if (total) *total = smem_warp[32];
  __syncthreads();
  return res;
}

struct LoadU64 {
  const unsigned long long* p;
  __device__ unsigned long long operator()(int64_t i) const { return p[i]; }
};
struct LoadPopc {
  const uint32_t* p;
  __device__ unsigned long long operator()(int64_t i) const { return (unsigned long long)__popc(p[i]); }
};

template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load load, int64_t count,
                                                                unsigned long long* partial) {
  pdl_wait();  // launched as a programmatic dependent
  __shared__ unsigned long long red[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long s = 0;
#pragma unroll 4
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < count) s += load(i);
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0ull;
    for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of `nparts` partial sums in place; total at [nparts].
__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* partial, int64_t nparts) {
  pdl_wait();  // launched as a programmatic dependent
  __shared__ unsigned long long sw[33];
  unsigned long long carry = 0;
  for (int64_t base = 0; base < nparts; base += 1024) {
    int64_t i = base + threadIdx.x;
    unsigned long long v = i < nparts ? partial[i] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan(v, sw, &tot);
    if (i < nparts) partial[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) partial[nparts] = carry;
}

template <class OutT>
struct StorePrefix {
  OutT* out;
  __device__ void operator()(int64_t i, unsigned long long run) const { out[i] = (OutT)run; }
  __device__ void total(int64_t count, unsigned long long t) const { out[count] = (OutT)t; }
};
// {word, popcount of the words before it}: one 8-byte read ranks a bit
struct StoreRanked {
  const uint32_t* words;
  uint2* out;
  __device__ void operator()(int64_t i, unsigned long long run) const {
    out[i] = make_uint2(words[i], (uint32_t)run);
  }
  __device__ void total(int64_t count, unsigned long long t) const { out[count] = make_uint2(0u, (uint32_t)t); }
};

// Shared-memory slot of tile item i: one pad slot per 16 items, so both the
// striped accesses and each thread's run of kScanItems hit distinct banks.
__device__ __forceinline__ int scan_slot(int i) { return i + (i >> 4); }

// Loads and stores are striped across the block (coalesced); a shared-memory
// transpose hands every thread kScanItems consecutive items to scan.
template <class Load, class Store>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(Load load, int64_t count,
                                                              const unsigned long long* partial,
                                                              Store store) {
  pdl_wait();  // launched as a programmatic dependent
  __shared__ unsigned long long sw[33];
  __shared__ unsigned long long sv[kScanTile + kScanTile / 16];
  const int64_t tile0 = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int local = k * kScanThreads + threadIdx.x;
    const int64_t i = tile0 + local;
    sv[scan_slot(local)] = i < count ? load(i) : 0ull;
  }
  __syncthreads();
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += sv[scan_slot(threadIdx.x * kScanItems + k)];
  unsigned long long ex = block_exclusive_scan(s, sw, (unsigned long long*)nullptr);
  unsigned long long run = ex + partial[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {  // each item becomes its exclusive prefix
    const int j = scan_slot(threadIdx.x * kScanItems + k);
    const unsigned long long t = sv[j];
    sv[j] = run;
    run += t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int local = k * kScanThreads + threadIdx.x;
    const int64_t i = tile0 + local;
    if (i < count) store(i, sv[scan_slot(local)]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) store.total(count, partial[gridDim.x]);
}

template <class Load, class Store>
static rst_status scan_impl(Load load, Store store, int64_t count, unsigned long long* tmp,
                            cudaStream_t s) {
  int64_t blocks = (count + kScanTile - 1) / kScanTile;
  if (blocks < 1) blocks = 1;
  RST_LAUNCH_PDL((k_scan_reduce<Load>), (unsigned)blocks, kScanThreads, 0, s)(load, count, tmp);
  RST_LAUNCH_PDL(k_scan_partials, 1, 1024, 0, s)(tmp, blocks);
  RST_LAUNCH_PDL((k_scan_down<Load, Store>), (unsigned)blocks, kScanThreads, 0, s)(load, count, tmp, store);
  RST_CUDA(cudaGetLastError());
  return RST_OK;
}

rst_status scan_exclusive_u64(const unsigned long long* in, unsigned long long* out, int64_t count,
                              unsigned long long* tmp, cudaStream_t s) {
  return scan_impl(LoadU64{in}, StorePrefix<unsigned long long>{out}, count, tmp, s);
}

rst_status scan_popcount_words(const uint32_t* words, uint32_t* out, int64_t count,
                               unsigned long long* tmp, cudaStream_t s) {
  return scan_impl(LoadPopc{words}, StorePrefix<uint32_t>{out}, count, tmp, s);
}

rst_status scan_popcount_ranked(const uint32_t* words, uint2* out, int64_t count,
                                unsigned long long* tmp, cudaStream_t s) {
  return scan_impl(LoadPopc{words}, StoreRanked{words, out}, count, tmp, s);
}

}  // namespace rst

extern "C" {

long long rst_launch_count(void) { return rst::g_launches.load(); }

int rst_last_stats(long long* out, int max) {
  int k = max < rst::STAT_COUNT ? max : rst::STAT_COUNT;
  for (int i = 0; i < k; ++i) out[i] = rst::g_stats[i];
  return k;
}

void rst_profile_enable(int on) {
  std::lock_guard<std::mutex> g(rst::call_lock());
  for (auto& m : rst::g_prof.marks) rst::g_prof.pool.push_back(m.second);
  rst::g_prof.marks.clear();
  rst::g_prof.on = on != 0;
}

void rst_profile_only(const char* names) {
  std::lock_guard<std::mutex> g(rst::call_lock());
  rst::g_prof.only.clear();
  if (!names) return;
  std::string cur;
  for (const char* c = names;; ++c) {
    if (*c == ',' || *c == '\0') {
      if (!cur.empty()) rst::g_prof.only.push_back(cur);
      cur.clear();
      if (*c == '\0') break;
    } else {
      cur.push_back(*c);
    }
  }
}

int rst_profile_read(float* ms_out, const char** names_out, int max_stages) {
  std::lock_guard<std::mutex> g(rst::call_lock());
  auto& marks = rst::g_prof.marks;
  int k = 0;
  if (!marks.empty()) cudaEventSynchronize(marks.back().second);
  for (size_t i = 1; i < marks.size() && k < max_stages; ++i, ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second);
    if (ms_out) ms_out[k] = ms;
    if (names_out) names_out[k] = marks[i].first;
  }
  for (auto& m : marks) rst::g_prof.pool.push_back(m.second);
  marks.clear();
  return k;
}

}  // extern "C"
