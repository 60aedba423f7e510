// Learned strategy selector: graph features, a 12-64-64-3 MLP (FP32) with
// hand-written forward, backward and Adam kernels, and the RST_AUTO choice.
//
// The paper compares BFS, CC+Euler and PR-RST and finds the winner depends on
// the graph's depth (Section IV-B); the selector predicts the log-time of each
// strategy from cheap features and picks the fastest, falling back to the
// depth-oblivious CC+Euler when the predicted margin is small.  No part of the
// paper prescribes this network; it is a deployment addition.
//
// Features (float, in this order), all computed on the device:
//   0 log2 n                       6 fraction of vertices with degree <= 2
//   1 log2 m (undirected edges)    7 log2 (1 + vertices reached in an 8-level BFS probe)
//   2 mean degree                  8 log2 ((1 + frontier at level 7) / (1 + frontier at level 3))
//   3 degree coefficient of var.   9 log2 eccentricity estimate from the probe
//   4 degree skewness             10 log2 (round-1 components / n) of the min-key hooking
//   5 log2 (1 + max degree)       11 fraction of the edges that survive one hook pass (their
//                                    ends lie in different round-1 components)
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

// Counts of the input that determine the features (device memory): degree
// moments, round-1 roots with edges, surviving edges, and the BFS probe's
// frontier sizes (filled in by the host loop that drives the probe).
struct SelRaw {
  double s1, s2, s3, le2;
  unsigned long long maxdeg, r1roots, survive;
  long long probe_levels, probe_finished, probe_reached, probe_last;
  long long frontier[8];
};

// Edges u < v whose ends lie in different round-1 components (R = round-1 root).
template <class OffT>
__global__ void k_sel_survive(const OffT* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                              const int32_t* __restrict__ R, unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ru = R[u];
    const int64_t hi = (int64_t)off[u + 1];
    for (int64_t j = (int64_t)off[u]; j < hi; ++j) {
      const int32_t v = col[j];
      if (v > (int32_t)u && (int64_t)v < n && R[v] != ru) ++c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// The twelve features from the raw counts (one thread).
__global__ void k_sel_assemble(int64_t n, int64_t A, const SelRaw* __restrict__ r, float* __restrict__ f) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double N = (double)(n > 0 ? n : 1);
  const double mu = r->s1 / N;
  const double var = r->s2 / N - mu * mu;
  const double sd = var > 0 ? sqrt(var) : 0.0;
  const double m3 = r->s3 / N - 3.0 * mu * (r->s2 / N) + 2.0 * mu * mu * mu;
  const double m = (double)(A / 2);
  f[0] = (float)log2(N);
  f[1] = (float)log2(m > 1 ? m : 1.0);
  f[2] = (float)mu;
  f[3] = (float)(mu > 0 ? sd / mu : 0.0);
  f[4] = (float)(sd > 0 ? m3 / (sd * sd * sd) : 0.0);
  f[5] = (float)log2(1.0 + (double)r->maxdeg);
  f[6] = (float)(r->le2 / N);
  const long long levels = r->probe_levels;
  const double reached = levels > 0 ? (double)r->probe_reached : 1.0;
  f[7] = (float)log2(1.0 + reached);
  const double f3 = levels > 3 ? (double)r->frontier[3] : 0.0;
  const double f7 = levels > 7 ? (double)r->frontier[7] : 0.0;
  f[8] = (float)log2((1.0 + f7) / (1.0 + f3));
  double ecc;
  if (levels == 0 || r->probe_finished) {
    ecc = (double)(levels > 0 ? levels : 1);
  } else {
    const double rest = N - reached;
    const double fr = (double)(r->probe_last > 0 ? r->probe_last : 1);
    ecc = (double)levels + (rest > 0 ? rest / fr : 0.0);
  }
  f[9] = (float)log2(1.0 + ecc);
  const double c1 = (double)(r->r1roots > 0 ? r->r1roots : 1);
  f[10] = (float)log2(c1 / N);
  f[11] = (float)(m > 0 ? (double)r->survive / m : 0.0);
}

struct FeatBufs {
  int32_t* parent;  // probe scratch
  int32_t* P;       // round-1 roots
  uint32_t* J;
  uint4* pairs;
  uint32_t* bits;
  SelRaw* raw;
  unsigned long long* cnt;  // round-1 tree-edge counter
  float* feat;              // 12 features
};

static FeatBufs feat_layout(Arena& ar, int64_t n, int64_t A) {
  FeatBufs b;
  b.parent = ar.take<int32_t>(n + 1);
  b.P = ar.take<int32_t>(n + 1);
  b.J = ar.take<uint32_t>(n + 1);
  b.pairs = ar.take<uint4>(n + 1);
  b.bits = ar.take<uint32_t>(A / 32 + 2);
  b.raw = ar.take<SelRaw>(1);
  b.cnt = ar.take<unsigned long long>(4);
  b.feat = ar.take<float>(16);
  return b;
}

static size_t feat_workspace_bytes(int64_t n, int64_t A) {
  Arena a;
  a.counting = true;
  feat_layout(a, n, A);
  return a.used + bfs_workspace_bytes(n) + 1024;
}

// Features of one graph into device memory (*feat_dev, 12 floats in the
// workspace); the BFS probe is the only host-driven part (it reads its
// frontier sizes back, 8 levels at most).
template <class OffT>
static rst_status features_impl(const OffT* off, const int32_t* col, int64_t n, int64_t A, int32_t root,
                                float** feat_dev, Arena& ar, cudaStream_t s) {
  FeatBufs b = feat_layout(ar, n, A);
  if (ar.used > ar.cap) return RST_ERR_OOM;
  RST_CUDA(cudaMemsetAsync(b.raw, 0, sizeof(SelRaw), s));
  RST_CUDA(cudaMemsetAsync(b.cnt, 0, 4 * sizeof(unsigned long long), s));
  RST_CUDA(cudaMemsetAsync(b.bits, 0, (A / 32 + 2) * sizeof(uint32_t), s));
  RST_LAUNCH(k_sel_degrees<OffT>, grid_for(n), kBlock, 0, s)(off, n, &b.raw->s1, &b.raw->maxdeg);
  RST_LAUNCH(k_sel_r1roots<OffT>, grid_for(n), kBlock, 0, s)(off, col, n, &b.raw->r1roots);
  RST_TRY(round1_forest<OffT>(off, col, n, b.P, b.J, b.pairs, b.bits, b.cnt, s));
  RST_LAUNCH(k_sel_survive<OffT>, grid_for(n), kBlock, 0, s)(off, col, n, b.P, &b.raw->survive);
  RST_CUDA(cudaGetLastError());
  BfsProbe probe;
  probe.max_levels = 8;
  const int bits = sizeof(OffT) == 8 ? 64 : 32;
  RST_TRY(bfs_probe_in(ar, off, bits, col, n, A, root, b.parent, &probe, s));
  // the probe's counts join the device record (pinned staging; the copy is
  // queued before any later read-back reuses the buffer)
  long long* stage = reinterpret_cast<long long*>(state().hostbuf + 256);
  stage[0] = probe.levels;
  stage[1] = probe.finished ? 1 : 0;
  stage[2] = probe.reached;
  stage[3] = probe.last_frontier;
  for (int i = 0; i < 8; ++i) stage[4 + i] = i < BfsProbe::kMax ? probe.frontier[i] : 0;
  RST_CUDA(cudaMemcpyAsync(&b.raw->probe_levels, stage, 12 * sizeof(long long), cudaMemcpyHostToDevice, s));
  RST_LAUNCH(k_sel_assemble, 1, 32, 0, s)(n, A, b.raw, b.feat);
  RST_CUDA(cudaGetLastError());
  *feat_dev = b.feat;
  return RST_OK;
}

static rst_status features_any(const void* off, int bits, const int32_t* col, int64_t n, int64_t m, int32_t root,
                               float** feat_dev, Arena& ar, cudaStream_t s) {
  if (bits == 32) return features_impl<int32_t>((const int32_t*)off, col, n, m, root, feat_dev, ar, s);
  return features_impl<int64_t>((const int64_t*)off, col, n, m, root, feat_dev, ar, s);
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

// gW[j][i] = sum_s dY[s][j] X[s][i]; gb[j] = sum_s dY[s][j].  One block per
// weight (blockIdx = j * (in + 1) + i, i == in: the bias): the block's threads
// stride over the batch and a fixed-order tree adds their partial sums, so the
// result is the same on every run.
constexpr int kWgradThreads = 128;
__global__ void __launch_bounds__(kWgradThreads) k_mlp_wgrad(const float* __restrict__ dY,
                                                             const float* __restrict__ X, int B, int in, int out,
                                                             float* __restrict__ gW, float* __restrict__ gb) {
  __shared__ float s_part[kWgradThreads / 32];
  const int64_t total = (int64_t)out * (in + 1);
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const int j = (int)(t / (in + 1)), i = (int)(t % (in + 1));
    float acc = 0.f;
    if (i < in) {
      for (int s = threadIdx.x; s < B; s += blockDim.x) acc = fmaf(dY[(int64_t)s * out + j], X[(int64_t)s * in + i], acc);
    } else {
      for (int s = threadIdx.x; s < B; s += blockDim.x) acc += dY[(int64_t)s * out + j];
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float sum = 0.f;
      for (int w = 0; w < kWgradThreads / 32; ++w) sum += s_part[w];
      if (i < in)
        gW[(int64_t)j * in + i] = sum;
      else
        gb[j] = sum;
    }
    __syncthreads();
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
  RST_LAUNCH(k_mlp_wgrad, kO * (kH + 1), kWgradThreads, 0, st)(s.dy, s.h2, B, kH, kO, G + kW3, G + kB3);
  RST_LAUNCH(k_mlp_dinput, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW3, s.dy, s.h2, B, kH, kO, s.dh2);
  RST_LAUNCH(k_mlp_wgrad, kH * (kH + 1), kWgradThreads, 0, st)(s.dh2, s.h1, B, kH, kH, G + kW2, G + kB2);
  RST_LAUNCH(k_mlp_dinput, grid_for((int64_t)B * kH), kBlock, 0, st)(P + kW2, s.dh2, s.h1, B, kH, kH, s.dh1);
  RST_LAUNCH(k_mlp_wgrad, kH * (kF + 1), kWgradThreads, 0, st)(s.dh1, X, B, kF, kH, G + kW1, G + kB1);
}

// ------------------------------------------------------------------ selector state

// The loaded model: network parameters, feature and target normalisation and
// the fallback margin.  The host keeps the master copy (rst_selector_load);
// each device gets its own copy before its first prediction after a load.
struct SelModel {
  float params[kParams];
  float xmean[kF], xstd[kF], ymean[kO], ystd[kO];
  float margin;
};
struct SelectorState {
  bool loaded = false;
  int version = 0;
  SelModel model;
};
static SelectorState g_sel;
constexpr int kSelMaxDev = 64;
static SelModel* g_sel_dev[kSelMaxDev] = {};
static int g_sel_dev_version[kSelMaxDev] = {};

// Inference of the loaded network on the device, one block per feature row:
// standardise, 12-64-64-3 with ReLU, un-standardise to predicted natural-log
// times (order BFS, CC+Euler, PR-RST), then pick the smallest and fall back to
// CC+Euler when the predicted gain of another strategy is below the margin.
__global__ void __launch_bounds__(kH) k_sel_infer(const SelModel* __restrict__ M, const float* __restrict__ feat,
                                                  int B, float* __restrict__ pred, int32_t* __restrict__ choice) {
  __shared__ float x[kF], h1[kH], h2[kH], y[kO];
  const int t = threadIdx.x;
  const float* P = M->params;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (t < kF) x[t] = (feat[(int64_t)b * kF + t] - M->xmean[t]) / M->xstd[t];
    __syncthreads();
    float a = P[kB1 + t];
    for (int i = 0; i < kF; ++i) a = fmaf(P[kW1 + t * kF + i], x[i], a);
    h1[t] = fmaxf(a, 0.f);
    __syncthreads();
    a = P[kB2 + t];
    for (int i = 0; i < kH; ++i) a = fmaf(P[kW2 + t * kH + i], h1[i], a);
    h2[t] = fmaxf(a, 0.f);
    __syncthreads();
    if (t < kO) {
      a = P[kB3 + t];
      for (int i = 0; i < kH; ++i) a = fmaf(P[kW3 + t * kH + i], h2[i], a);
      y[t] = a * M->ystd[t] + M->ymean[t];
      if (pred) pred[(int64_t)b * kO + t] = y[t];
    }
    __syncthreads();
    if (t == 0 && choice) {
      int best = 1;
      for (int k = 0; k < kO; ++k)
        if (y[k] < y[best]) best = k;
      if (best != 1 && y[1] - y[best] < M->margin) best = 1;  // small predicted gain: CC+Euler
      choice[b] = best == 0 ? (int32_t)RST_BFS : (best == 1 ? (int32_t)RST_CC_EULER : (int32_t)RST_PR_RST);
    }
    __syncthreads();
  }
}

// The current device's copy of the loaded model (uploaded after each load).
static rst_status model_on_device(const SelModel** out, cudaStream_t s) {
  int dev = 0;
  RST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kSelMaxDev) return RST_ERR_UNSUPPORTED;
  if (!g_sel_dev[dev]) RST_CUDA(cudaMalloc(&g_sel_dev[dev], sizeof(SelModel)));
  if (g_sel_dev_version[dev] != g_sel.version) {
    RST_CUDA(cudaMemcpyAsync(g_sel_dev[dev], &g_sel.model, sizeof(SelModel), cudaMemcpyHostToDevice, s));
    RST_CUDA(cudaStreamSynchronize(s));
    g_sel_dev_version[dev] = g_sel.version;
  }
  *out = g_sel_dev[dev];
  return RST_OK;
}

void release_selector() {
  for (int d = 0; d < kSelMaxDev; ++d)
    if (g_sel_dev[d]) {
      cudaFree(g_sel_dev[d]);
      g_sel_dev[d] = nullptr;
      g_sel_dev_version[d] = 0;
    }
}

// Features, inference and the choice of one graph, all on the device; only
// the choice and the three predictions come back to the host.
static rst_status select_impl(const void* off, int bits, const int32_t* cols, int64_t n, int64_t m, int32_t root,
                              rst_strategy* choice_out, float* pred_out, cudaStream_t s) {
  RST_TRY(ensure_workspace(feat_workspace_bytes(n, m) + 1024));
  RST_TRY(reset_device_error(s));
  const SelModel* M = nullptr;
  RST_TRY(model_on_device(&M, s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  float* fd = nullptr;
  RST_TRY(features_any(off, bits, cols, n, m, root, &fd, ar, s));
  float* pd = ar.take<float>(kO);
  int32_t* cd = ar.take<int32_t>(1);
  if (ar.used > ar.cap) return RST_ERR_OOM;
  RST_LAUNCH(k_sel_infer, 1, kH, 0, s)(M, fd, 1, pd, cd);
  RST_CUDA(cudaGetLastError());
  unsigned long long* hb = st.hostbuf + 16;  // word 0 receives the status word
  RST_CUDA(cudaMemcpyAsync(hb, pd, kO * sizeof(float), cudaMemcpyDeviceToHost, s));
  RST_CUDA(cudaMemcpyAsync(hb + 2, cd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RST_TRY(read_device_error(s));
  float pred[kO];
  int32_t c = 0;
  std::memcpy(pred, hb, sizeof(pred));
  std::memcpy(&c, hb + 2, sizeof(c));
  *choice_out = (rst_strategy)c;
  if (pred_out)
    for (int k = 0; k < kO; ++k) pred_out[k] = pred[k];
  return RST_OK;
}

rst_strategy select_strategy_host(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                                  int32_t root, cudaStream_t s) {
  if (!g_sel.loaded) return RST_CC_EULER;
  rst_strategy c = RST_CC_EULER;
  if (select_impl(off, offsets_bits, cols, n, m, root, &c, nullptr, s) != RST_OK) return RST_CC_EULER;
  return c;
}

}  // namespace rst

using namespace rst;

extern "C" {

rst_status rst_selector_features(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n,
                                 int64_t m, int32_t root, float* features_out, rst_stream_t stream) {
  if (!features_out || (offsets_bits != 32 && offsets_bits != 64) || n <= 0 || root < 0 || root >= n)
    return RST_ERR_INVALID_ARG;
  if (!csr_offsets || (m > 0 && !csr_cols) || n >= ((int64_t)1 << 30) || m >= ((int64_t)1 << 32))
    return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RST_TRY(ensure_workspace(feat_workspace_bytes(n, m)));
  RST_TRY(reset_device_error(s));
  DeviceState& st = state();
  Arena ar{st.ws, st.ws_cap, 0, false};
  float* fd = nullptr;
  RST_TRY(features_any(csr_offsets, offsets_bits, csr_cols, n, m, root, &fd, ar, s));
  // features land after the word that read_device_error fills with the status
  RST_CUDA(cudaMemcpyAsync(st.hostbuf + 16, fd, kF * sizeof(float), cudaMemcpyDeviceToHost, s));
  RST_TRY(read_device_error(s));
  std::memcpy(features_out, st.hostbuf + 16, kF * sizeof(float));
  return RST_OK;
}

rst_status rst_selector_load(const float* params, const float* norm, float margin) {
  if (!params || !norm) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  SelModel& M = g_sel.model;
  std::memcpy(M.params, params, sizeof(M.params));
  std::memcpy(M.xmean, norm, sizeof(float) * kF);
  std::memcpy(M.xstd, norm + kF, sizeof(float) * kF);
  std::memcpy(M.ymean, norm + 2 * kF, sizeof(float) * kO);
  std::memcpy(M.ystd, norm + 2 * kF + kO, sizeof(float) * kO);
  for (int i = 0; i < kF; ++i)
    if (!(M.xstd[i] > 0)) M.xstd[i] = 1.f;
  for (int k = 0; k < kO; ++k)
    if (!(M.ystd[k] > 0)) M.ystd[k] = 1.f;
  M.margin = margin;
  g_sel.loaded = true;
  g_sel.version += 1;
  return RST_OK;
}

rst_status rst_selector_predict(const float* features, int batch, float* pred_out, int32_t* choice_out,
                                rst_stream_t stream) {
  if (!features || batch <= 0 || (!pred_out && !choice_out)) return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  if (!g_sel.loaded) return RST_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const SelModel* M = nullptr;
  RST_TRY(model_on_device(&M, s));
  const int grid = batch < device_info().sms * 16 ? batch : device_info().sms * 16;
  RST_LAUNCH(k_sel_infer, grid, kH, 0, s)(M, features, batch, pred_out, choice_out);
  RST_CUDA(cudaGetLastError());
  RST_CUDA(cudaStreamSynchronize(s));
  return RST_OK;
}

rst_status rst_select(const void* csr_offsets, int offsets_bits, const int32_t* csr_cols, int64_t n, int64_t m,
                      int32_t root, rst_strategy* choice_out, float* pred_log_time_out, rst_stream_t stream) {
  if (!choice_out || (offsets_bits != 32 && offsets_bits != 64) || n <= 0 || root < 0 || root >= n)
    return RST_ERR_INVALID_ARG;
  if (!csr_offsets || (m > 0 && !csr_cols) || n >= ((int64_t)1 << 30) || m >= ((int64_t)1 << 32))
    return RST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(call_lock());
  if (!g_sel.loaded) {
    *choice_out = RST_CC_EULER;
    if (pred_log_time_out)
      for (int k = 0; k < kO; ++k) pred_log_time_out[k] = NAN;
    return RST_OK;
  }
  return select_impl(csr_offsets, offsets_bits, csr_cols, n, m, root, choice_out, pred_log_time_out,
                     reinterpret_cast<cudaStream_t>(stream));
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
  if (std::strcmp(key, "pr_levels_per_launch") == 0) {
    if (value < 1 || value > 3) return RST_ERR_INVALID_ARG;
    t.pr_levels = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "euler_block") == 0) {
    if (value != 128 && value != 256 && value != 512) return RST_ERR_INVALID_ARG;
    t.euler_block = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "giant_share_pct") == 0) {
    if (value < 0 || value > 101) return RST_ERR_INVALID_ARG;
    t.giant_pct = (int)value;
    return RST_OK;
  }
  if (std::strcmp(key, "insert_walk_limit") == 0) {
    if (value < 0 || value > (1LL << 30)) return RST_ERR_INVALID_ARG;
    t.insert_walk_limit = value;
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
  else if (std::strcmp(key, "insert_walk_limit") == 0) *value = t.insert_walk_limit;
  else if (std::strcmp(key, "euler_block") == 0) *value = t.euler_block;
  else if (std::strcmp(key, "pr_levels_per_launch") == 0) *value = t.pr_levels;
  else if (std::strcmp(key, "giant_share_pct") == 0) *value = t.giant_pct;
  else return RST_ERR_INVALID_ARG;
  return RST_OK;
}

}  // extern "C"
