// rst_build_batch: thousands of independent graphs as one disjoint union.
//
// The paper blames BFS's cost on high-diameter graphs on the sequence of
// per-level kernel launches and synchronisations (Section I and Section IV-B);
// many small graphs processed one call each pay the same fixed per-launch cost
// once per graph.  Here the graphs of a batch are renumbered into one union
// graph (global ids = per-graph vertex offset + local id) and the whole batch
// runs through a single pipeline: the union's components are exactly the
// graphs' components, the minimum spanning forest of the union is the union of
// the graphs' forests, and the per-graph roots become the requested roots of
// their components.  Parents are translated back to local ids at the end.
#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

namespace {

// Largest g in [0, G) with tab[g] <= x (tab non-decreasing, tab[0] = 0).
__device__ __forceinline__ int32_t seg_of(const int64_t* __restrict__ tab, int32_t G, int64_t x) {
  int32_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (tab[mid] <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Global offsets from the concatenated per-graph offset arrays (graph g's
// n_g + 1 local offsets start at index vtx_off[g] + g).
template <class InT, class OutT>
__global__ void k_batch_offsets(const InT* __restrict__ loff, const int64_t* __restrict__ vtx_off,
                                const int64_t* __restrict__ arc_off, int32_t G, int64_t N, int64_t A,
                                OutT* __restrict__ goff) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= N;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (x == N) {
      goff[N] = (OutT)A;
      continue;
    }
    const int32_t g = seg_of(vtx_off, G, x);
    const int64_t i = x - vtx_off[g];
    goff[x] = (OutT)(arc_off[g] + (int64_t)loff[vtx_off[g] + g + i]);
  }
}

__global__ void k_batch_cols(const int32_t* __restrict__ lcol, const int64_t* __restrict__ vtx_off,
                             const int64_t* __restrict__ arc_off, int32_t G, int64_t A,
                             int32_t* __restrict__ gcol, uint32_t* status) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = seg_of(arc_off, G, a);
    const int64_t ng = vtx_off[g + 1] - vtx_off[g];
    const int32_t c = lcol[a];
    if (c < 0 || c >= ng) {
      raise_error(status, DERR_INDEX);
      gcol[a] = (int32_t)vtx_off[g];
    } else {
      gcol[a] = (int32_t)(vtx_off[g] + c);
    }
  }
}

__global__ void k_batch_roots(const int32_t* __restrict__ roots, const int64_t* __restrict__ vtx_off,
                              int32_t G, int32_t* __restrict__ groots, uint32_t* status) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int64_t ng = vtx_off[g + 1] - vtx_off[g];
    const int32_t r = roots[g];
    if (ng == 0) {
      groots[g] = -1;
    } else if (r < 0 || r >= ng) {
      raise_error(status, DERR_INDEX);
      groots[g] = -1;
    } else {
      groots[g] = (int32_t)(vtx_off[g] + r);
    }
  }
}

__global__ void k_batch_rootof(const int32_t* __restrict__ groots, int32_t G, const int32_t* __restrict__ labels,
                               int32_t* __restrict__ rootof) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int32_t r = groots[g];
    if (r >= 0) rootof[labels[r]] = r;
  }
}

__global__ void k_batch_localize(int32_t* __restrict__ parent, const int64_t* __restrict__ vtx_off, int32_t G,
                                 int64_t N) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = seg_of(vtx_off, G, x);
    parent[x] = (int32_t)(parent[x] - vtx_off[g]);
  }
}

__global__ void k_fill_i32_b(int32_t* p, int64_t count, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

template <class GOffT>
rst_status batch_run(const void* loff, int offsets_bits, const int32_t* lcol, const int64_t* vtx_off,
                     const int64_t* arc_off, int32_t G, const int32_t* roots, rst_strategy strategy,
                     int32_t* parent, int64_t N, int64_t A, cudaStream_t s) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256 + 256; };
  size_t ws = al((N + 1) * sizeof(GOffT)) + al(A * 4) + al(N * 4) * 2 + al(G * 4);
  if (strategy == RST_CC_EULER)
    ws += cc_workspace_bytes<GOffT>(N, A) + euler_cc_workspace_bytes(N, A, N, N / 2 + 1);
  else
    ws += bfs_workspace_bytes(N);
  RST_TRY(ensure_workspace(ws));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  GOffT* goff = ar.take<GOffT>(N + 1);
  int32_t* gcol = ar.take<int32_t>(A);
  int32_t* labels = ar.take<int32_t>(N);
  int32_t* rootof = ar.take<int32_t>(N);
  int32_t* groots = ar.take<int32_t>(G);
  if (!groots) return RST_ERR_OOM;
  uint32_t* status = st.status;
  prof_mark(s, "batch_start");
  if (offsets_bits == 32)
    RST_LAUNCH((k_batch_offsets<int32_t, GOffT>), grid_for(N + 1), kBlock, 0, s)(
        (const int32_t*)loff, vtx_off, arc_off, G, N, A, goff);
  else
    RST_LAUNCH((k_batch_offsets<int64_t, GOffT>), grid_for(N + 1), kBlock, 0, s)(
        (const int64_t*)loff, vtx_off, arc_off, G, N, A, goff);
  if (A > 0) RST_LAUNCH(k_batch_cols, grid_for(A), kBlock, 0, s)(lcol, vtx_off, arc_off, G, A, gcol, status);
  RST_LAUNCH(k_batch_roots, grid_for(G), kBlock, 0, s)(roots, vtx_off, G, groots, status);
  prof_mark(s, "batch_union");
  RST_CUDA(cudaGetLastError());
  const int gbits = sizeof(GOffT) == 8 ? 64 : 32;
  if (strategy == RST_BFS) {
    RST_TRY(bfs_multi_in(ar, goff, gbits, gcol, N, A, groots, G, parent, s));
  } else {
    CcOut cc;
    RST_TRY(cc_run<GOffT>(ar, goff, gcol, N, A, -1, labels, &cc, s));
    RST_LAUNCH(k_fill_i32_b, grid_for(N), kBlock, 0, s)(rootof, N, -1);
    RST_LAUNCH(k_batch_rootof, grid_for(G), kBlock, 0, s)(groots, G, labels, rootof);
    cc.rootof = rootof;
    RST_TRY(euler_root_cc<GOffT>(ar, goff, N, A, -1, &cc, parent, nullptr, s));
  }
  RST_LAUNCH(k_batch_localize, grid_for(N), kBlock, 0, s)(parent, vtx_off, G, N);
  prof_mark(s, "batch_end");
  RST_CUDA(cudaGetLastError());
  return read_device_error(s);
}

}  // namespace
}  // namespace rst

extern "C" rst_status rst_build_batch(const void* packed_offsets, int offsets_bits, const int32_t* packed_cols,
                                      const int64_t* graph_vtx_off, const int64_t* graph_arc_off,
                                      int32_t num_graphs, const int32_t* roots, rst_strategy strategy,
                                      int32_t* parent_out, rst_stream_t stream) {
  using namespace rst;
  if (num_graphs < 0 || (offsets_bits != 32 && offsets_bits != 64)) return RST_ERR_INVALID_ARG;
  if (num_graphs == 0) return RST_OK;
  if (!packed_offsets || !graph_vtx_off || !graph_arc_off || !roots || !parent_out) return RST_ERR_INVALID_ARG;
  if (strategy == RST_AUTO) strategy = RST_CC_EULER;
  if (strategy != RST_CC_EULER && strategy != RST_BFS) return RST_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(call_lock());
  RST_TRY(ensure_workspace(0));
  // totals (host)
  int64_t tot[2] = {0, 0};
  RST_CUDA(cudaMemcpyAsync(host_scratch(16), graph_vtx_off + num_graphs, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaMemcpyAsync(static_cast<char*>(host_scratch(16)) + 8, graph_arc_off + num_graphs, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaStreamSynchronize(s));
  std::memcpy(tot, host_scratch(16), sizeof(tot));
  const int64_t N = tot[0], A = tot[1];
  if (N < 0 || A < 0) return RST_ERR_INVALID_ARG;
  if (N >= ((int64_t)1 << 30) || A >= ((int64_t)1 << 32)) return RST_ERR_UNSUPPORTED;
  if (N == 0) return RST_OK;
  if (A > 0 && !packed_cols) return RST_ERR_INVALID_ARG;
  if (A < ((int64_t)1 << 31))
    return batch_run<int32_t>(packed_offsets, offsets_bits, packed_cols, graph_vtx_off, graph_arc_off, num_graphs,
                              roots, strategy, parent_out, N, A, s);
  return batch_run<int64_t>(packed_offsets, offsets_bits, packed_cols, graph_vtx_off, graph_arc_off, num_graphs,
                            roots, strategy, parent_out, N, A, s);
}
