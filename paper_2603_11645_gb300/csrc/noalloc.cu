// rst_build_noalloc: CC+Euler rooted spanning tree without any allocation.
//
// Some callers cannot allocate device memory: a serving process or an
// embedding runtime that reserves its whole device-memory budget at start-up
// (a pool this library cannot draw from), and hosts whose allocator must not
// be entered from the calling thread.  For them this entry point carves its
// whole workspace out of a fixed device array defined in this file, so it
// never calls cudaMalloc, cudaFree, cudaMallocHost or any allocating library
// routine, and creates no event, stream or graph (the contraction rounds run
// from the host, one round at a time, reading the round count back into a
// static host buffer).  The first call on a device looks up the array's
// device address (cudaGetSymbolAddress, with that device current); that
// first call should come before any stream capture begins.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library holds it (kNoAllocScratchBytes + 256 bytes) until the process
// exits.  All calls on a device share it and it keeps the previous call's
// contents; the pipeline clears everything that must start at zero.  Calls
// whose work overlaps on the GPU (two streams, or several host threads
// without waiting) race on the array; host-side calls are serialised.
#include "pipeline.cuh"

namespace rst {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int64_t kNoAllocMaxVertices = int64_t(1) << 16;  // 65,536
constexpr int64_t kNoAllocMaxArcs = int64_t(1) << 19;      // 524,288

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) uint32_t g_noalloc_status[64];

namespace {

constexpr int kMaxDev = 64;
struct NoAllocSlot {
  bool ready = false;
  DeviceState st;
};
NoAllocSlot g_slots[kMaxDev];
unsigned long long g_host_words[kMaxDev][kHostBufWords];  // static host buffer for readbacks

// Per-device set-up, with that device current: resolve the device addresses of
// the fixed arrays (the host-side names are only stand-ins).
rst_status noalloc_setup(int dev, DeviceState** out) {
  NoAllocSlot& slot = g_slots[dev];
  if (!slot.ready) {
    void* scratch = nullptr;
    void* status = nullptr;
    RST_CUDA(cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
    RST_CUDA(cudaGetSymbolAddress(&status, g_noalloc_status));
    slot.st.ws = static_cast<char*>(scratch);
    slot.st.ws_cap = kNoAllocScratchBytes;
    slot.st.status = static_cast<uint32_t*>(status);
    slot.st.hostbuf = g_host_words[dev];
    slot.ready = true;
  }
  *out = &slot.st;
  return RST_OK;
}

struct OverrideGuard {
  explicit OverrideGuard(DeviceState* st) { set_state_override(st); }
  ~OverrideGuard() { set_state_override(nullptr); }
};

template <class OffT>
rst_status noalloc_build(const OffT* off, const int32_t* cols, int64_t n, int64_t m, int32_t root,
                         int32_t* parent, cudaStream_t s) {
  const size_t need = cc_workspace_bytes<OffT>(n, m) + euler_cc_workspace_bytes(n, m, n, n / 2 + 1);
  if (need > kNoAllocScratchBytes) return RST_ERR_UNSUPPORTED;
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  CcOut cc;
  RST_TRY(cc_run<OffT>(ar, off, cols, n, m, root, nullptr, &cc, s));
  RST_TRY(euler_root_cc<OffT>(ar, off, n, m, root, &cc, parent, nullptr, s));
  return read_device_error(s);
}

}  // namespace
}  // namespace rst

extern "C" rst_status rst_build_noalloc(const void* csr_offsets, int offsets_bits,
                                        const int32_t* csr_cols, int64_t n, int64_t m,
                                        int32_t root, int32_t* parent_out, rst_stream_t stream) {
  using namespace rst;
  if (n < 0 || m < 0 || (offsets_bits != 32 && offsets_bits != 64)) return RST_ERR_INVALID_ARG;
  if (n > kNoAllocMaxVertices || m > kNoAllocMaxArcs) return RST_ERR_UNSUPPORTED;
  if (n == 0) return RST_OK;
  if (!csr_offsets || (m > 0 && !csr_cols) || !parent_out || root < 0 || root >= n)
    return RST_ERR_INVALID_ARG;
  int dev = 0;
  RST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return RST_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(call_lock());
  DeviceState* st = nullptr;
  RST_TRY(noalloc_setup(dev, &st));
  OverrideGuard guard(st);
  if (offsets_bits == 32)
    return noalloc_build<int32_t>((const int32_t*)csr_offsets, csr_cols, n, m, root, parent_out, s);
  return noalloc_build<int64_t>((const int64_t*)csr_offsets, csr_cols, n, m, root, parent_out, s);
}
