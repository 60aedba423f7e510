// extern "C" entry points of librst.so (declared in include/rst.h).
#include <cstring>

#include "pipeline.cuh"
#include "strategies.cuh"

using namespace rst;

namespace {

struct CallGuard {
  std::unique_lock<std::mutex> lk;
  CallGuard() : lk(call_lock()) {}
};

rst_status check_graph(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m) {
  if (n < 0 || m < 0) return RST_ERR_INVALID_ARG;
  if (offsets_bits != 32 && offsets_bits != 64) return RST_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 30)) return RST_ERR_UNSUPPORTED;
  if (m >= ((int64_t)1 << 32)) return RST_ERR_UNSUPPORTED;
  if (offsets_bits == 32 && m >= ((int64_t)1 << 31)) return RST_ERR_INVALID_ARG;
  if (n > 0 && !off) return RST_ERR_INVALID_ARG;
  if (m > 0 && !cols) return RST_ERR_INVALID_ARG;
  return RST_OK;
}

rst_status begin(size_t ws_bytes, cudaStream_t s, Arena* ar) {
  RST_TRY(ensure_workspace(ws_bytes));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  ar->base = st.ws;
  ar->cap = st.ws_cap;
  ar->used = 0;
  return RST_OK;
}

template <class OffT>
rst_status build_cc_euler(const OffT* off, const int32_t* cols, int64_t n, int64_t m, int32_t root,
                          int32_t* parent, uint32_t* rank_out, cudaStream_t s) {
  const size_t ws = cc_workspace_bytes<OffT>(n, m) + euler_cc_workspace_bytes(n, m, n, n / 2 + 1);
  Arena ar;
  prof_mark(s, "start");
  RST_TRY(begin(ws, s, &ar));
  CcOut cc;
  RST_TRY(cc_run<OffT>(ar, off, cols, n, m, root, nullptr, &cc, s, /*prefetch_euler=*/true));
  RST_TRY(euler_root_cc<OffT>(ar, off, n, m, root, &cc, parent, rank_out, s));
  rst_status st = read_device_error(s);
  prof_mark(s, "end");
  return st;
}

template <class OffT>
rst_status build_cc_fast(const OffT* off, const int32_t* cols, int64_t n, int64_t m, int32_t root,
                         int32_t* parent, cudaStream_t s) {
  const size_t ws = ccfast_workspace_bytes<OffT>(n, m) + euler_cc_workspace_bytes(n, m, n, n / 2 + 1);
  Arena ar;
  prof_mark(s, "start");
  RST_TRY(begin(ws, s, &ar));
  CcOut cc;
  RST_TRY(ccfast_run<OffT>(ar, off, cols, n, m, root, nullptr, &cc, s));
  RST_TRY(euler_root_cc<OffT>(ar, off, n, m, root, &cc, parent, nullptr, s));
  rst_status st = read_device_error(s);
  prof_mark(s, "end");
  return st;
}

__global__ void k_pairs_to_uv(int64_t T, const uint4* __restrict__ pairs, int32_t* __restrict__ uv) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = pairs[t];
    const int32_t a = (int32_t)r.z, b = (int32_t)r.w;
    uv[2 * t] = a < b ? a : b;
    uv[2 * t + 1] = a < b ? b : a;
  }
}

template <class OffT>
rst_status cc_only(const OffT* off, const int32_t* cols, int64_t n, int64_t m, int32_t* labels,
                   int32_t* tree_uv, int64_t* num_tree, cudaStream_t s) {
  const size_t ws = cc_workspace_bytes<OffT>(n, m);
  Arena ar;
  RST_TRY(begin(ws, s, &ar));
  CcOut cc;
  RST_TRY(cc_run<OffT>(ar, off, cols, n, m, -1, labels, &cc, s));
  if (tree_uv && cc.T > 0) {
    RST_LAUNCH(k_pairs_to_uv, grid_for(cc.T), kBlock, 0, s)(cc.T, cc.pairs, tree_uv);
    RST_CUDA(cudaGetLastError());
  }
  if (num_tree) *num_tree = cc.T;
  return read_device_error(s);
}

}  // namespace

extern "C" {

const char* rst_status_string(rst_status s) {
  switch (s) {
    case RST_OK: return "ok";
    case RST_ERR_INVALID_ARG: return "invalid argument";
    case RST_ERR_OOM: return "out of device memory";
    case RST_ERR_CUDA: return "CUDA error";
    case RST_ERR_NOT_CONVERGED: return "iteration bound exceeded";
    case RST_ERR_TIMEOUT: return "timeout";
    case RST_ERR_UNSUPPORTED: return "unsupported size or strategy";
    case RST_ERR_DEVICE: return "error detected on the device (malformed input)";
  }
  return "unknown status";
}

int rst_version(void) { return 100; }

rst_status rst_build(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n,
                     int64_t m, int32_t root, rst_strategy strategy, int32_t* parent_out,
                     rst_stream_t stream) {
  RST_TRY(check_graph(csr_offsets, offsets_bits, csr_cols, n, m));
  if (n == 0) return RST_OK;
  if (!parent_out || root < 0 || root >= n) return RST_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  if (strategy == RST_AUTO) strategy = select_strategy_host(csr_offsets, offsets_bits, csr_cols, n, m, root, s);
  switch (strategy) {
    case RST_CC_EULER:
      if (offsets_bits == 32)
        return build_cc_euler<int32_t>((const int32_t*)csr_offsets, csr_cols, n, m, root, parent_out,
                                       nullptr, s);
      return build_cc_euler<int64_t>((const int64_t*)csr_offsets, csr_cols, n, m, root, parent_out,
                                     nullptr, s);
    case RST_BFS:
      return run_bfs(csr_offsets, offsets_bits, csr_cols, n, m, root, parent_out, nullptr, s);
    case RST_BFS_DEVICE:
      return run_bfs_device(csr_offsets, offsets_bits, csr_cols, n, m, root, parent_out, nullptr, s, false);
    case RST_BFS_PERSISTENT:
      return run_bfs_device(csr_offsets, offsets_bits, csr_cols, n, m, root, parent_out, nullptr, s, true);
    case RST_PR_RST:
      return run_prrst(csr_offsets, offsets_bits, csr_cols, n, m, root, parent_out, s);
    case RST_CC_FAST:
      if (offsets_bits == 32)
        return build_cc_fast<int32_t>((const int32_t*)csr_offsets, csr_cols, n, m, root, parent_out, s);
      return build_cc_fast<int64_t>((const int64_t*)csr_offsets, csr_cols, n, m, root, parent_out, s);
    default:
      return RST_ERR_INVALID_ARG;
  }
}

rst_status rst_cc(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n,
                  int64_t m, int32_t* labels_out, int32_t* tree_uv_out, int64_t* num_tree_edges_out,
                  rst_stream_t stream) {
  RST_TRY(check_graph(csr_offsets, offsets_bits, csr_cols, n, m));
  if (n == 0) {
    if (num_tree_edges_out) *num_tree_edges_out = 0;
    return RST_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  if (offsets_bits == 32)
    return cc_only<int32_t>((const int32_t*)csr_offsets, csr_cols, n, m, labels_out, tree_uv_out,
                            num_tree_edges_out, s);
  return cc_only<int64_t>((const int64_t*)csr_offsets, csr_cols, n, m, labels_out, tree_uv_out,
                          num_tree_edges_out, s);
}

rst_status rst_euler_root(int64_t n, const int32_t* tree_uv, int64_t num_tree_edges, int32_t root,
                          int32_t* parent_out, int32_t* rank_out, rst_stream_t stream) {
  if (n < 0 || num_tree_edges < 0 || num_tree_edges >= (n > 0 ? n : 1)) return RST_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 30)) return RST_ERR_UNSUPPORTED;
  if (n == 0) return RST_OK;
  if (!parent_out || root < 0 || root >= n) return RST_ERR_INVALID_ARG;
  if (num_tree_edges > 0 && !tree_uv) return RST_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  Arena ar;
  RST_TRY(begin(euler_edges_workspace_bytes(n, num_tree_edges), s, &ar));
  RST_TRY(euler_root_edges(ar, n, tree_uv, num_tree_edges, root, parent_out,
                           reinterpret_cast<uint32_t*>(rank_out), s));
  return read_device_error(s);
}

rst_status rst_verify(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n,
                      int64_t m, int32_t root, const int32_t* parent, int32_t* verdict_out,
                      rst_stream_t stream) {
  RST_TRY(check_graph(csr_offsets, offsets_bits, csr_cols, n, m));
  if (!verdict_out) return RST_ERR_INVALID_ARG;
  if (n == 0) {
    *verdict_out = RST_VERDICT_VALID;
    return RST_OK;
  }
  if (!parent) return RST_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  return run_verify(csr_offsets, offsets_bits, csr_cols, n, m, root, parent, verdict_out, s);
}

rst_status rst_bcc(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n, int64_t m,
                   uint32_t* block_out, uint8_t* cut_out, int64_t* num_blocks_out, rst_stream_t stream) {
  RST_TRY(check_graph(csr_offsets, offsets_bits, csr_cols, n, m));
  if (m > 0 && !block_out) return RST_ERR_INVALID_ARG;
  if (n == 0) {
    if (num_blocks_out) *num_blocks_out = 0;
    return RST_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  Arena ar;
  if (offsets_bits == 32) {
    RST_TRY(begin(bcc_workspace_bytes<int32_t>(n, m), s, &ar));
    RST_TRY(bcc_run<int32_t>(ar, (const int32_t*)csr_offsets, csr_cols, n, m, block_out, cut_out,
                             num_blocks_out, s));
  } else {
    RST_TRY(begin(bcc_workspace_bytes<int64_t>(n, m), s, &ar));
    RST_TRY(bcc_run<int64_t>(ar, (const int64_t*)csr_offsets, csr_cols, n, m, block_out, cut_out,
                             num_blocks_out, s));
  }
  return read_device_error(s);
}

rst_status rst_insert_edges(int64_t n, int32_t* parent, const int32_t* new_uv, int64_t k, int32_t root,
                            unsigned int flags, rst_stream_t stream) {
  if (n <= 0 || n >= ((int64_t)1 << 30) || k < 0) return RST_ERR_INVALID_ARG;
  if (!parent || (k > 0 && !new_uv) || root < 0 || root >= n) return RST_ERR_INVALID_ARG;
  if (flags & ~(unsigned int)RST_INSERT_CANONICAL) return RST_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  return run_prrst_insert(n, parent, new_uv, k, root, (flags & RST_INSERT_CANONICAL) != 0, s);
}

rst_status rst_tree_depth(const int32_t* parent, int64_t n, int32_t* depth_out, int64_t* max_out,
                          rst_stream_t stream) {
  if (n < 0 || n >= ((int64_t)1 << 30)) return RST_ERR_INVALID_ARG;
  if (n > 0 && !parent) return RST_ERR_INVALID_ARG;
  if (n == 0) {
    if (max_out) *max_out = 0;
    return RST_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CallGuard g;
  RST_TRY(ensure_workspace(depth_workspace_bytes(n)));
  RST_TRY(reset_device_error(s));
  return tree_depth(parent, n, depth_out, max_out, s);
}

rst_status rst_shutdown(void) {
  CallGuard g;
  destroy_round_graphs();
  destroy_bfs_graphs();
  release_selector();
  DeviceState& st = state();
  if (st.ws) cudaFree(st.ws);
  if (st.status) cudaFree(st.status);
  if (st.hostbuf) cudaFreeHost(st.hostbuf);
  if (st.readback) cudaEventDestroy(st.readback);
  st = DeviceState{};
  return RST_OK;
}

}  // extern "C"
