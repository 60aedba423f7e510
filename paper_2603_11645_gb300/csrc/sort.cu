// Stable LSD radix sort of 64-bit keys (hand-written, 8-bit digits).
//
// Used to put tree arcs into lexicographic (src, dst) order (Section III-D:
// "generate 2(N-1) directed edges and lexicographically sort them").  Each
// pass: per-tile digit histograms (digit-major in global memory), one
// exclusive scan over them, then a stable scatter in which every tile ranks
// its keys in index order with warp match + per-warp digit counters.
#include "pipeline.cuh"

namespace rst {

constexpr int kSortThreads = 256;
constexpr int kSortSub = 16;                       // sub-rounds per tile
constexpr int kSortTile = kSortThreads * kSortSub;  // keys per tile
constexpr int kRadix = 256;

static int64_t sort_tiles(int64_t count) { return (count + kSortTile - 1) / kSortTile; }

size_t radix_sort_workspace_bytes(int64_t count) {
  const int64_t tiles = sort_tiles(count);
  const int64_t hist = tiles * kRadix;
  size_t b = 0;
  b += ((count * 8 + 255) / 256) * 256 + 256;              // key buffer
  b += ((hist * 8 + 255) / 256) * 256 + 256;               // histograms
  b += ((scan_tmp_words(hist) * 8 + 255) / 256) * 256 + 256;
  return b;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ keys, int64_t count,
                                                            int shift, unsigned long long* __restrict__ hist,
                                                            int64_t tiles) {
  __shared__ uint32_t h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortSub; ++k) {
    const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
    if (i < count) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * tiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ in, int64_t count,
                                                               int shift,
                                                               const unsigned long long* __restrict__ offs,
                                                               int64_t tiles, uint64_t* __restrict__ out) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned long long run[kRadix];   // next output slot per digit
  __shared__ uint32_t wc[kWarps][kRadix];      // per-warp digit counts, then starts
  __shared__ uint32_t tot[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] = offs[(int64_t)d * tiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortSub; ++k) {
    const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
    const bool valid = i < count;
    const uint64_t key = valid ? in[i] : 0ull;
    const int d = valid ? (int)((key >> shift) & (kRadix - 1)) : kRadix;  // kRadix: padding
    for (int j = threadIdx.x; j < kWarps * kRadix; j += blockDim.x) (&wc[0][0])[j] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int lrank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lrank == 0) wc[warp][d] = (uint32_t)__popc(peers);
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
      uint32_t acc = 0;
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t t = wc[w][dd];
        wc[w][dd] = acc;
        acc += t;
      }
      tot[dd] = acc;
    }
    __syncthreads();
    if (valid) out[run[d] + wc[warp][d] + lrank] = key;
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) run[dd] += tot[dd];
    __syncthreads();
  }
}

rst_status radix_sort_keys(Arena& ar, uint64_t* keys, int64_t count, int key_bits, cudaStream_t s) {
  if (count <= 1) return RST_OK;
  const int64_t tiles = sort_tiles(count);
  const int64_t hist_n = tiles * kRadix;
  uint64_t* alt = ar.take<uint64_t>(count);
  unsigned long long* hist = ar.take<unsigned long long>(hist_n + 1);
  unsigned long long* tmp = ar.take<unsigned long long>(scan_tmp_words(hist_n));
  if (!alt || !hist || !tmp) return RST_ERR_OOM;
  uint64_t* src = keys;
  uint64_t* dst = alt;
  int passes = 0;
  for (int shift = 0; shift < key_bits; shift += 8, ++passes) {
    RST_LAUNCH(k_sort_hist, (unsigned)tiles, kSortThreads, 0, s)(src, count, shift, hist, tiles);
    RST_TRY(scan_exclusive_u64(hist, hist, hist_n, tmp, s));
    RST_LAUNCH(k_sort_scatter, (unsigned)tiles, kSortThreads, 0, s)(src, count, shift, hist, tiles, dst);
    std::swap(src, dst);
  }
  RST_CUDA(cudaGetLastError());
  if (src != keys) RST_CUDA(cudaMemcpyAsync(keys, src, count * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  return RST_OK;
}

}  // namespace rst
