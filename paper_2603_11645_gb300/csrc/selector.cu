// Learned strategy selector: graph features, a 12-64-64-3 MLP (FP32) with
// hand-written forward, backward and Adam kernels, and the RST_AUTO choice.
//
// The paper compares BFS, CC+Euler and PR-RST and finds the winner depends on
// the graph's depth (Section IV-B); the selector predicts the log-time of each
// strategy from cheap features and picks the fastest, falling back to the
// depth-oblivious CC+Euler when the predicted margin is small.  No part of the
// paper prescribes this network; it is a deployment addition.
//
// Features (float, in this order):
//   0 log2 n                       6 fraction of vertices with degree <= 2
//   1 log2 m (undirected edges)    7 log2 (1 + vertices reached in an 8-level BFS probe)
//   2 mean degree                  8 log2 ((1 + frontier at level 7) / (1 + frontier at level 3))
//   3 degree coefficient of var.   9 log2 eccentricity estimate from the probe
//   4 degree skewness             10 log2 (round-1 components / n) of the min-key hooking
//   5 log2 (1 + max degree)       11 fraction of vertices the probe reached
#include <cmath>

#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

constexpr int kF = 12, kH = 64, kO = 3;
constexpr int kW1 = 0, kB1 = kW1 + kH * kF, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kO * kH, kParams = kB3 + kO;  // 5187

static_assert(kParams == 5187, "parameter count");

// ------------------------------------------------------------------ features

// Degree moments: sum d, sum d^2, sum d^3 (double), max d, #(d <= 2).
template <class OffT>
__global__ void k_sel_degrees(const OffT* __restrict__ off, int64_t n, double* __restrict__ acc,
                              unsigned long long* __restrict__ imax) {
  double s1 = 0, s2 = 0, s3 = 0, le2 = 0;
  unsigned long long mx = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)(off[v + 1] - off[v]);
    s1 += d;
    s2 += d * d;
    s3 += d * d * d;
    le2 += d <= 2.0 ? 1.0 : 0.0;
    const unsigned long long di = (unsigned long long)(off[v + 1] - off[v]);
    mx = di > mx ? di : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    s3 += __shfl_down_sync(0xffffffffu, s3, o);
    le2 += __shfl_down_sync(0xffffffffu, le2, o);
    const unsigned long long m2 = __shfl_down_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s1);
    atomicAdd(&acc[1], s2);
    atomicAdd(&acc[2], s3);
    atomicAdd(&acc[3], le2);
    atomicMax(imax, mx);
  }
}

// Round-1 components of the min-key hooking that still have edges: vertex u
// is such a root iff its first neighbour's first neighbour is u and u is the
// smaller of the two.
template <class OffT>
__global__ void k_sel_r1roots(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                              unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = (int64_t)off[u], hi = (int64_t)off[u + 1];
    while (j < hi && col[j] == (int32_t)u) ++j;
    if (j >= hi) continue;
    const int32_t v0 = col[j];
    if (v0 < 0 || v0 >= n || v0 < (int32_t)u) continue;
    int64_t k = (int64_t)off[v0], h2 = (int64_t)off[v0 + 1];
    while (k < h2 && col[k] == v0) ++k;
    if (k < h2 && col[k] == (int32_t)u) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

struct FeatureRaw {
  double s1, s2, s3, le2;
  unsigned long long maxdeg, r1roots;
};

static void assemble_features(int64_t n, int64_t A, const FeatureRaw& r, const BfsProbe& p, float* f) {
  const double N = (double)(n > 0 ? n : 1);
  const double mu = r.s1 / N;
  const double var = r.s2 / N - mu * mu;
  const double sd = var > 0 ? std::sqrt(var) : 0.0;
  const double m3 = r.s3 / N - 3.0 * mu * (r.s2 / N) + 2.0 * mu * mu * mu;
  const double m = (double)(A / 2);
  f[0] = (float)std::log2(N);
  f[1] = (float)std::log2(m > 1 ? m : 1.0);
  f[2] = (float)mu;
  f[3] = (float)(mu > 0 ? sd / mu : 0.0);
  f[4] = (float)(sd > 0 ? m3 / (sd * sd * sd) : 0.0);
  f[5] = (float)std::log2(1.0 + (double)r.maxdeg);
  f[6] = (float)(r.le2 / N);
  const double reached = p.levels > 0 ? (double)p.reached : 1.0;
  f[7] = (float)std::log2(1.0 + reached);
  const double f3 = p.levels > 3 ? (double)p.frontier[3] : 0.0;
  const double f7 = p.levels > 7 ? (double)p.frontier[7] : 0.0;
  f[8] = (float)std::log2((1.0 + f7) / (1.0 + f3));
  double ecc;
  if (p.levels == 0 || p.finished) {
    ecc = (double)(p.levels > 0 ? p.levels : 1);
  } else {
    const double rest = N - reached;
    const double fr = (double)(p.last_frontier > 0 ? p.last_frontier : 1);
    ecc = (double)p.levels + (rest > 0 ? rest / fr : 0.0);
  }
  f[9] = (float)std::log2(1.0 + ecc);
  const double c1 = (double)(r.r1roots > 0 ? r.r1roots : 1);
  f[10] = (float)std::log2(c1 / N);
  f[11] = (float)(reached / N);
}

template <class OffT>
static rst_status features_impl(const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                                float* feat_host, cudaStream_t s) {
  const size_t ws = bfs_workspace_bytes(n) + (((size_t)n * 4 + 255) / 256 * 256 + 256) + 1024;
  RST_TRY(ensure_workspace(ws));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  int32_t* scratch_parent = ar.take<int32_t>(n);
  double* acc = ar.take<double>(4);
  unsigned long long* ic = ar.take<unsigned long long>(2);
  if (!acc || !ic) return RST_ERR_OOM;
  RST_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
  RST_CUDA(cudaMemsetAsync(ic, 0, 2 * sizeof(unsigned long long), s));
  RST_LAUNCH(k_sel_degrees<OffT>, grid_for(n), kBlock, 0, s)(off, n, acc, ic);
  RST_LAUNCH(k_sel_r1roots<OffT>, grid_for(n), kBlock, 0, s)(off, col, n, ic + 1);
  RST_CUDA(cudaGetLastError());
  FeatureRaw raw{};
  char* hs = static_cast<char*>(host_scratch(64));
  RST_CUDA(cudaMemcpyAsync(hs, acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaMemcpyAsync(hs + 32, ic, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaStreamSynchronize(s));
  std::memcpy(&raw.s1, hs, 8);
  std::memcpy(&raw.s2, hs + 8, 8);
  std::memcpy(&raw.s3, hs + 16, 8);
  std::memcpy(&raw.le2, hs + 24, 8);
  std::memcpy(&raw.maxdeg, hs + 32, 8);
  std::memcpy(&raw.r1roots, hs + 40, 8);
  BfsProbe probe;
  probe.max_levels = 8;
  const int bits = sizeof(OffT) == 8 ? 64 : 32;
  RST_TRY(bfs_probe_in(ar, off, bits, col, n, A, root, scratch_parent, &probe, s));
  assemble_features(n, A, raw, probe, feat_host);
  return read_device_error(s);
}

static rst_status features_any(const void* off, int bits, const int32_t* col, int64_t n, int64_t m, int32_t root,
                               float* feat, cudaStream_t s) {
  if (bits == 32) return features_impl<int32_t>((const int32_t*)off, col, n, m, root, feat, s);
  return features_impl<int64_t>((const int64_t*)off, col, n, m, root, feat, s);
}

// ------------------------------------------------------------------ MLP kernels
// Row-major weights: W1[64][12], W2[64][64], W3[3][64]; batch-major activations.

__global__ void k_mlp_layer(const float* __restrict__ W, const float* __restrict__ b, const float* __restrict__ X,
                            int B, int in, int out, int relu, float* __restrict__ Y) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * out;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / out), j = (int)(t % out);
    float acc = b[j];
    const float* x = X + (int64_t)s * in;
    const float* w = W + (int64_t)j * in;
    for (int i = 0; i < in; ++i) acc = fmaf(w[i], x[i], acc);
    Y[t] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// dY = 2 (Y - T) / (B * 3); also accumulates the loss.
__global__ void k_mlp_dout(const float* __restrict__ Y, const float* __restrict__ T, int B, float* __restrict__ dY,
                           float* loss) {
  float l = 0.f;
  const float scale = 1.f / (float)(B * kO);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * kO;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[t] - T[t];
    dY[t] = 2.f * d * scale;
    l += d * d * scale;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// dX[s][i] = sum_j W[j][i] dY[s][j], masked by the ReLU of H (H = the layer input).
__global__ void k_mlp_dinput(const float* __restrict__ W, const float* __restrict__ dY, const float* __restrict__ H,
                             int B, int in, int out, float* __restrict__ dX) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * in;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / in), i = (int)(t % in);
    float acc = 0.f;
    for (int j = 0; j < out; ++j) acc = fmaf(W[(int64_t)j * in + i], dY[(int64_t)s * out + j], acc);
    dX[t] = H[t] > 0.f ? acc : 0.f;
  }
}

// gW[j][i] = sum_s dY[s][j] X[s][i]; gb[j] = sum_s dY[s][j].  One thread per weight.
__global__ void k_mlp_wgrad(const float* __restrict__ dY, const float* __restrict__ X, int B, int in, int out,
                            float* __restrict__ gW, float* __restrict__ gb) {
  const int64_t total = (int64_t)out * (in + 1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / (in + 1)), i = (int)(t % (in + 1));
    float acc = 0.f;
    if (i < in) {
      for (int s = 0; s < B; ++s) acc = fmaf(dY[(int64_t)s * out + j], X[(int64_t)s * in + i], acc);
      gW[(int64_t)j * in + i] = acc;
    } else {
      for (int s = 0; s < B; ++s) acc += dY[(int64_t)s * out + j];
      gb[j] = acc;
    }
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int count, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

struct MlpScratch {
  float *h1, *h2, *y, *dy, *dh2, *dh1;
};

static size_t mlp_scratch_bytes(int B) {
  return (size_t)B * (kH * 4 + kO * 2) * 4 + 6 * 256;
}

static MlpScratch mlp_scratch(Arena& ar, int B) {
  MlpScratch s;
  s.h1 = ar.take<float>((size_t)B * kH);
  s.h2 = ar.take<float>((size_t)B * kH);
  s.y = ar.take<float>((size_t)B * kO);
  s.dy = ar.take<float>((size_t)B * kO);
  s.dh2 = ar.take<float>((size_t)B * kH);
  s.dh1 = ar.take<float>((size_t)B * kH);
  return s;
}

static void mlp_forward(const float* P, const float* X, int B, MlpScratch& s, float* Y, cudaStream_t st) {
  RST_LAUNCH(k_mlp_layer, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW1, P + kB1, X, B, kF, kH, 1, s.h1);
  RST_LAUNCH(k_mlp_layer, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW2, P + kB2, s.h1, B, kH, kH, 1, s.h2);
  RST_LAUNCH(k_mlp_layer, grid_for((int64_t)B * kO), kBlock, 0, st)(P + kW3, P + kB3, s.h2, B, kH, kO, 0, Y);
}

static void mlp_grad(const float* P, const float* X, const float* T, int B, MlpScratch& s, float* G, float* loss,
                     cudaStream_t st) {
  mlp_forward(P, X, B, s, s.y, st);
  RST_LAUNCH(k_mlp_dout, grid_for((int64_t)B * kO), kBlock, 0, st)(s.y, T, B, s.dy, loss);
  RST_LAUNCH(k_mlp_wgrad, grid_for((int64_t)kO * (kH + 1)), kBlock, 0, st)(s.dy, s.h2, B, kH, kO, G + kW3, G + kB3);
  RST_LAUNCH(k_mlp_dinput, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW3, s.dy, s.h2, B, kH, kO, s.dh2);
  RST_LAUNCH(k_mlp_wgrad, grid_for((int64_t)kH * (kH + 1)), kBlock, 0, st)(s.dh2, s.h1, B, kH, kH, G + kW2, G + kB2);
  RST_LAUNCH(k_mlp_dinput, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW2, s.dh2, s.h1, B, kH, kH, s.dh1);
  RST_LAUNCH(k_mlp_wgrad, grid_for((int64_t)kH * (kF + 1)), kBlock, 0, st)(s.dh1, X, B, kF, kH, G + kW1, G + kB1);
}

// ------------------------------------------------------------------ selector state

struct SelectorState {
  bool loaded = false;
  float params[kParams];
  float xmean[kF], xstd[kF], ymean[kO], ystd[kO];
  float margin = 0.f;
};
static SelectorState g_sel;

// Host forward pass of the loaded network (12 features: inference is tiny and
// host-side; the training kernels above run on the GPU).
static void sel_predict(const float* f, float* pred) {
  float x[kF], h1[kH], h2[kH];
  for (int i = 0; i < kF; ++i) x[i] = (f[i] - g_sel.xmean[i]) / g_sel.xstd[i];
  const float* P = g_sel.params;
  for (int j = 0; j < kH; ++j) {
    float a = P[kB1 + j];
    for (int i = 0; i < kF; ++i) a += P[kW1 + j * kF + i] * x[i];
    h1[j] = a > 0 ? a : 0;
  }
  for (int j = 0; j < kH; ++j) {
    float a = P[kB2 + j];
    for (int i = 0; i < kH; ++i) a += P[kW2 + j * kH + i] * h1[i];
    h2[j] = a > 0 ? a : 0;
  }
  for (int k = 0; k < kO; ++k) {
    float a = P[kB3 + k];
    for (int i = 0; i < kH; ++i) a += P[kW3 + k * kH + i] * h2[i];
    pred[k] = a * g_sel.ystd[k] + g_sel.ymean[k];
  }
}

// Output order of the network: BFS, CC+Euler, PR-RST.
static rst_strategy sel_choose(const float* pred) {
  int best = 1;
  for (int k = 0; k < kO; ++k)
    if (pred[k] < pred[best]) best = k;
  if (best != 1 && pred[1] - pred[best] < g_sel.margin) best = 1;  // small margin: CC+Euler
  return best == 0 ? RST_BFS : (best == 1 ? RST_CC_EULER : RST_PR_RST);
}

rst_strategy select_strategy_host(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                                  int32_t root, cudaStream_t s) {
  if (!g_sel.loaded) return RST_CC_EULER;
  float f[kF], pred[kO];
  if (features_any(off, offsets_bits, cols, n, m, root, f, s) != RST_OK) return RST_CC_EULER;
  sel_predict(f, pred);
  return sel_choose(pred);
}

}  // namespace rst

using namespace rst;

extern "C" {

rst_status rst_selector_features(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n,
                                 int64_t m, int32_t root, float* features_out, rst_stream_t stream) {
  if (!features_out || (offsets_bits != 32 && offsets_bits != 64) || n <= 0 || root < 0 || root >= n)
    return RST_ERR_INVALID_ARG;
  if (!csr_offsets || (m > 0 && !csr_cols)) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  return features_any(csr_offsets, offsets_bits, csr_cols, n, m, root, features_out,
                      reinterpret_cast<cudaStream_t>(stream));
}

rst_status rst_selector_load(const float* params, const float* norm, float margin) {
  if (!params || !norm) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  std::memcpy(g_sel.params, params, sizeof(g_sel.params));
  std::memcpy(g_sel.xmean, norm, sizeof(float) * kF);
  std::memcpy(g_sel.xstd, norm + kF, sizeof(float) * kF);
  std::memcpy(g_sel.ymean, norm + 2 * kF, sizeof(float) * kO);
  std::memcpy(g_sel.ystd, norm + 2 * kF + kO, sizeof(float) * kO);
  for (int i = 0; i < kF; ++i)
    if (!(g_sel.xstd[i] > 0)) g_sel.xstd[i] = 1.f;
  for (int k = 0; k < kO; ++k)
    if (!(g_sel.ystd[k] > 0)) g_sel.ystd[k] = 1.f;
  g_sel.margin = margin;
  g_sel.loaded = true;
  return RST_OK;
}

rst_status rst_select(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n, int64_t m,
                      int32_t root, rst_strategy* choice_out, float* pred_log_time_out, rst_stream_t stream) {
  if (!choice_out || (offsets_bits != 32 && offsets_bits != 64) || n <= 0 || root < 0 || root >= n)
    return RST_ERR_INVALID_ARG;
  if (!csr_offsets || (m > 0 && !csr_cols)) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  if (!g_sel.loaded) {
    *choice_out = RST_CC_EULER;
    if (pred_log_time_out)
      for (int k = 0; k < kO; ++k) pred_log_time_out[k] = NAN;
    return RST_OK;
  }
  float f[kF], pred[kO];
  RST_TRY(features_any(csr_offsets, offsets_bits, csr_cols, n, m, root, f, reinterpret_cast<cudaStream_t>(stream)));
  sel_predict(f, pred);
  *choice_out = sel_choose(pred);
  if (pred_log_time_out)
    for (int k = 0; k < kO; ++k) pred_log_time_out[k] = pred[k];
  return RST_OK;
}

rst_status rst_mlp_forward(const float* params, const float* X, int batch, float* Y, rst_stream_t stream) {
  if (!params || !X || !Y || batch <= 0) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RST_TRY(ensure_workspace(mlp_scratch_bytes(batch)));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  MlpScratch sc = mlp_scratch(ar, batch);
  if (!sc.dh1) return RST_ERR_OOM;
  mlp_forward(params, X, batch, sc, Y, s);
  RST_CUDA(cudaGetLastError());
  RST_CUDA(cudaStreamSynchronize(s));
  return RST_OK;
}

rst_status rst_mlp_loss_grad(const float* params, const float* X, const float* T, int batch, float* grad,
                             float* loss_out, rst_stream_t stream) {
  if (!params || !X || !T || !grad || batch <= 0) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RST_TRY(ensure_workspace(mlp_scratch_bytes(batch)));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  MlpScratch sc = mlp_scratch(ar, batch);
  if (!sc.dh1) return RST_ERR_OOM;
  if (loss_out) RST_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(float), s));
  mlp_grad(params, X, T, batch, sc, grad, loss_out, s);
  RST_CUDA(cudaGetLastError());
  RST_CUDA(cudaStreamSynchronize(s));
  return RST_OK;
}

rst_status rst_mlp_adam(float* params, const float* grad, float* m, float* v, int count, int step, float lr,
                        float beta1, float beta2, float eps, rst_stream_t stream) {
  if (!params || !grad || !m || !v || count <= 0 || step <= 0) return RST_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  RST_LAUNCH(k_mlp_adam, grid_for(count), kBlock, 0, s)(params, grad, m, v, count, lr, beta1, beta2, eps, c1, c2);
  RST_CUDA(cudaGetLastError());
  RST_CUDA(cudaStreamSynchronize(s));
  return RST_OK;
}

rst_status rst_mlp_train(float* params, const float* X, const float* T, int batch, int epochs, float lr,
                         float* adam_m, float* adam_v, float* loss_hist, rst_stream_t stream) {
  if (!params || !X || !T || !adam_m || !adam_v || batch <= 0 || epochs <= 0) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RST_TRY(ensure_workspace(mlp_scratch_bytes(batch) + kParams * 4 + 512));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  MlpScratch sc = mlp_scratch(ar, batch);
  float* G = ar.take<float>(kParams);
  if (!G) return RST_ERR_OOM;
  if (loss_hist) RST_CUDA(cudaMemsetAsync(loss_hist, 0, sizeof(float) * epochs, s));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int e = 1; e <= epochs; ++e) {
    mlp_grad(params, X, T, batch, sc, G, loss_hist ? loss_hist + (e - 1) : nullptr, s);
    const float c1 = 1.f - powf(b1, (float)e), c2 = 1.f - powf(b2, (float)e);
    RST_LAUNCH(k_mlp_adam, grid_for(kParams), kBlock, 0, s)(params, G, adam_m, adam_v, kParams, lr, b1, b2, eps, c1,
                                                            c2);
  }
  RST_CUDA(cudaGetLastError());
  RST_CUDA(cudaStreamSynchronize(s));
  return RST_OK;
}

rst_status rst_set_option(const char* key, long long value) {
  if (!key) return RST_ERR_INVALID_ARG;
  if (std::strcmp(key, "bfs_max_levels") == 0) {
    if (value < 0) return RST_ERR_INVALID_ARG;
    set_bfs_max_levels(value);
    return RST_OK;
  }
  Tuning& t = tuning();
  if (std::strcmp(key, "lr_spacing") == 0) {
    for (int sh = 4; sh <= 9; ++sh)
      if (value == (1LL << sh)) {
        t.lr_shift = sh;
        return RST_OK;
      }
    return RST_ERR_INVALID_ARG;
  }
  if (std::strcmp(key, "round_blocks_per_sm") == 0) {
    if (value < 1 || value > 16) return RST_ERR_INVALID_ARG;
    t.round_bps = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "bfs_device_blocks_per_sm") == 0) {
    if (value < 1 || value > 8) return RST_ERR_INVALID_ARG;
    tuning().bfsd_bps = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "bfs_persistent_blocks_per_sm") == 0) {
    if (value < 1 || value > 8) return RST_ERR_INVALID_ARG;
    tuning().bfsp_bps = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "bfs_bottom_up_divisor") == 0) {
    if (value < 1 || value > 1000000) return RST_ERR_INVALID_ARG;
    t.bfs_bu_div = (int)value;
    return RST_OK;
  }
  return RST_ERR_INVALID_ARG;
}

rst_status rst_get_option(const char* key, long long* value) {
  if (!key || !value) return RST_ERR_INVALID_ARG;
  const Tuning& t = tuning();
  if (std::strcmp(key, "bfs_max_levels") == 0) *value = get_bfs_max_levels();
  else if (std::strcmp(key, "lr_spacing") == 0) *value = 1LL << t.lr_shift;
  else if (std::strcmp(key, "round_blocks_per_sm") == 0) *value = t.round_bps;
  else if (std::strcmp(key, "bfs_bottom_up_divisor") == 0) *value = t.bfs_bu_div;
  else if (std::strcmp(key, "bfs_device_blocks_per_sm") == 0) *value = t.bfsd_bps;
  else if (std::strcmp(key, "bfs_persistent_blocks_per_sm") == 0) *value = t.bfsp_bps;
  else return RST_ERR_INVALID_ARG;
  return RST_OK;
}

}  // extern "C"
