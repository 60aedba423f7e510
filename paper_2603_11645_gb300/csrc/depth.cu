// Depth of every vertex of a rooted forest (the tree-shape comparison of
// Section IV-B and Fig. 2: connectivity-based trees are deeper than BFS trees).
//
// Pointer jumping with distances: anc[v] starts as parent[v] and dist[v] as
// 1 (0 at a root, parent[v] == v); a round sets anc'[v] = anc[anc[v]] and
// dist'[v] = dist[v] + dist[anc[v]].  After round k, anc[v] is v's ancestor
// 2^k levels up or its root, so ceil(log2(height)) + 1 rounds settle every
// vertex.  Rounds read one buffer and write the other (no in-place races);
// a round that moved no pointer ends the loop.  A parent array with a cycle
// never settles; after ceil(log2 n) + 1 rounds the call reports it.
#include <cstring>

#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

__global__ void k_depth_init(int64_t n, const int32_t* __restrict__ parent, int32_t* __restrict__ anc,
                             int32_t* __restrict__ dist, int32_t* bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = parent[v];
    if (p < 0 || (int64_t)p >= n) {
      *bad = 1;
      p = (int32_t)v;  // treated as a root so later rounds stay in bounds
    }
    anc[v] = p;
    dist[v] = p == (int32_t)v ? 0 : 1;
  }
}

__global__ void k_depth_round(int64_t n, const int32_t* __restrict__ anc, const int32_t* __restrict__ dist,
                              int32_t* __restrict__ anc2, int32_t* __restrict__ dist2, int32_t* moved) {
  bool any = false;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = anc[v];
    const int32_t aa = anc[a];
    anc2[v] = aa;
    dist2[v] = (int32_t)((uint32_t)dist[v] + (uint32_t)dist[a]);  // wraps only on a cycle
    any = any || aa != a;
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *moved = 1;
}

__global__ void k_depth_max(int64_t n, const int32_t* __restrict__ dist, int32_t* mx) {
  int32_t best = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    best = max(best, dist[v]);
  for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, d));
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(mx, best);
}

size_t depth_workspace_bytes(int64_t n) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  return 4 * al((size_t)n * 4) + al(64);
}

rst_status tree_depth(const int32_t* parent, int64_t n, int32_t* depth_out, int64_t* max_out,
                      cudaStream_t s) {
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  int32_t* a0 = ar.take<int32_t>(n);
  int32_t* d0 = ar.take<int32_t>(n);
  int32_t* a1 = ar.take<int32_t>(n);
  int32_t* d1 = depth_out ? depth_out : ar.take<int32_t>(n);
  int32_t* flags = ar.take<int32_t>(4);  // bad, moved, max
  if (!a0 || !d0 || !a1 || !d1 || !flags) return RST_ERR_OOM;
  const int g = grid_for(n);
  int32_t h[3] = {0, 0, 0};
  auto read_flags = [&]() -> rst_status {
    RST_CUDA(cudaMemcpyAsync(st.hostbuf, flags, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RST_CUDA(cudaStreamSynchronize(s));
    std::memcpy(h, st.hostbuf, 3 * sizeof(int32_t));
    return RST_OK;
  };
  RST_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int32_t), s));
  RST_LAUNCH(k_depth_init, g, kBlock, 0, s)(n, parent, a0, d0, flags);
  int limit = 2;
  while (((int64_t)1 << limit) < n) ++limit;
  bool settled = false;
  for (int r = 0; r <= limit; ++r) {
    RST_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int32_t), s));
    RST_LAUNCH(k_depth_round, g, kBlock, 0, s)(n, a0, d0, a1, d1, flags + 1);
    RST_CUDA(cudaGetLastError());
    std::swap(a0, a1);
    std::swap(d0, d1);
    RST_TRY(read_flags());
    if (h[0]) return RST_ERR_INVALID_ARG;
    if (!h[1]) {
      settled = true;
      break;
    }
  }
  if (!settled) return RST_ERR_NOT_CONVERGED;  // a cycle: some pointer never reaches a root
  // after the swap d0 holds the final distances
  if (depth_out && d0 != depth_out)
    RST_CUDA(cudaMemcpyAsync(depth_out, d0, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  RST_LAUNCH(k_depth_max, g, kBlock, 0, s)(n, d0, flags + 2);
  RST_CUDA(cudaGetLastError());
  RST_TRY(read_flags());
  if (max_out) *max_out = h[2];
  return RST_OK;
}

}  // namespace rst
