// Load-balanced traversal of every (row, arc) pair of a CSR graph.
//
// The rows' end offsets and the arc indices are merged into one sequence of
// n + A items (a merge path); each block takes a tile of kMpTile consecutive
// items and each thread kMpItems of them, so rows of any degree (a 4-neighbour
// mesh or an R-MAT hub with millions of arcs) cost the same per item.
#pragma once

#include "common.cuh"

namespace rst {

constexpr int kMpThreads = 256;
constexpr int kMpItems = 8;
constexpr int kMpTile = kMpThreads * kMpItems;

// Number of row-end items that precede diagonal `diag` of the merge of
// row ends (off[1..n]) with arc indices (0..A-1).
template <class OffT>
__device__ __forceinline__ int64_t mp_search(const OffT* __restrict__ off, int64_t n, int64_t A,
                                             int64_t diag) {
  int64_t lo = diag - A > 0 ? diag - A : 0;
  int64_t hi = diag < n ? diag : n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)off[mid + 1] <= diag - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Calls f(it, is_arc, row, arc) for it = 0..kMpItems-1 per thread per tile,
// then f.end_tile().  Every thread of the block makes the same calls (is_arc =
// false for row-end and padding items), so f may use warp- and block-
// collective operations; `it` is a compile-time index after unrolling.
// Grid-stride over tiles; blockDim.x must be kMpThreads.
template <class OffT, class F>
__device__ __forceinline__ void csr_for_each_arc(const OffT* __restrict__ off, int64_t n,
                                                 int64_t A, F& f) {
  __shared__ OffT s_rowend[kMpTile + 1];
  __shared__ int64_t s_split[2];
  const int64_t total = n + A;
  for (int64_t tile = blockIdx.x; tile * kMpTile < total; tile += gridDim.x) {
    const int64_t d0 = tile * kMpTile;
    const int64_t d1 = (d0 + kMpTile < total) ? d0 + kMpTile : total;
    if (threadIdx.x < 2) s_split[threadIdx.x] = mp_search(off, n, A, threadIdx.x == 0 ? d0 : d1);
    __syncthreads();
    const int64_t r0 = s_split[0], r1 = s_split[1];
    const int64_t a0 = d0 - r0, a1 = d1 - r1;
    const int nrows = (int)(r1 - r0);
    for (int k = threadIdx.x; k < nrows; k += blockDim.x) s_rowend[k] = off[r0 + k + 1];
    __syncthreads();
    const int64_t span = d1 - d0;
    int64_t td = (int64_t)threadIdx.x * kMpItems;
    if (td > span) td = span;
    int lo = (int)(td - (a1 - a0) > 0 ? td - (a1 - a0) : 0);
    int hi = (int)(td < nrows ? td : nrows);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if ((int64_t)s_rowend[mid] <= a0 + (td - mid - 1))
        lo = mid + 1;
      else
        hi = mid;
    }
    int64_t row = r0 + lo;
    int64_t arc = a0 + (td - lo);
#pragma unroll
    for (int it = 0; it < kMpItems; ++it) {
      const bool valid = td + it < span;
      bool is_arc = false;
      const int64_t my_row = row, my_arc = arc;
      if (valid) {
        const int lr = (int)(row - r0);
        if (lr < nrows && (int64_t)s_rowend[lr] <= arc) {
          ++row;
        } else {
          is_arc = true;
          ++arc;
        }
      }
      f(it, is_arc, my_row, my_arc);
    }
    f.end_tile();
    __syncthreads();
  }
}

// ------------------------------------------------------------------ arc tiles
// Arc-centric traversal: a block takes kArcTile consecutive arc positions and
// learns the row of every arc from one shared-memory max-scan (each row that
// starts inside the tile marks its first position; the running maximum of the
// marks is the row).  Threads then read arcs with fully coalesced loads and
// independent gathers, which suits the light rows of meshes and the heavy rows
// of power-law graphs alike.
constexpr int kArcThreads = 256;
constexpr int kArcPer = 8;
constexpr int kArcTile = kArcThreads * kArcPer;

// Last row r in [0, n) with off[r] <= a (the row holding arc a).
template <class OffT>
__device__ __forceinline__ int64_t row_of_arc(const OffT* __restrict__ off, int64_t n, int64_t a) {
  int64_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)off[mid] <= a)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// tile_row[t] = row holding arc t * kArcTile (t <= tiles; the last entry is
// n - 1 or the row of the last arc).  One thread per tile, all in parallel.
template <class OffT>
__global__ void k_arc_tile_rows(const OffT* __restrict__ off, int64_t n, int64_t A, int64_t tiles,
                                int32_t* __restrict__ tile_row) {
  pdl_wait();  // launched as a programmatic dependent
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t * kArcTile < A ? t * kArcTile : A - 1;
    tile_row[t] = (int32_t)row_of_arc(off, n, a < 0 ? 0 : a);
  }
}

// Fills s_row[i] with the row of arc a0 + i for i < cnt, given r0 = the row
// of arc a0 and r1 >= the row of arc a0 + cnt - 1 (from k_arc_tile_rows).
// Call from all threads of a kArcThreads block; s_row must be 16-byte
// aligned.  Ends with __syncthreads().
template <class OffT>
__device__ __forceinline__ void arc_tile_rows(const OffT* __restrict__ off, int64_t n, int64_t a0,
                                              int cnt, int32_t* s_row, int64_t r0, int64_t r1) {
  __shared__ int32_t s_warp[kArcThreads / 32];
  for (int i = threadIdx.x; i < kArcTile; i += kArcThreads) s_row[i] = -1;
  __syncthreads();
  for (int64_t r = r0 + 1 + threadIdx.x; r <= r1; r += kArcThreads) {
    const int64_t pos = (int64_t)off[r] - a0;
    if (pos >= 0 && pos < cnt) atomicMax(&s_row[pos], (int32_t)r);
  }
  if (threadIdx.x == 0) atomicMax(&s_row[0], (int32_t)r0);
  __syncthreads();
  // inclusive max-scan: kArcPer consecutive entries per thread (two 16-byte
  // shared loads, free of bank conflicts), then across threads
  static_assert(kArcPer == 8, "the scan reads two int4 per thread");
  int32_t v[kArcPer];
  {
    const int4 lo4 = reinterpret_cast<const int4*>(s_row)[2 * threadIdx.x];
    const int4 hi4 = reinterpret_cast<const int4*>(s_row)[2 * threadIdx.x + 1];
    v[0] = lo4.x; v[1] = lo4.y; v[2] = lo4.z; v[3] = lo4.w;
    v[4] = hi4.x; v[5] = hi4.y; v[6] = hi4.z; v[7] = hi4.w;
  }
  int32_t run = -1;
#pragma unroll
  for (int k = 0; k < kArcPer; ++k) {
    run = max(run, v[k]);
    v[k] = run;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x = max(x, y);
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  int32_t carry = -1;
  for (int w = 0; w < warp; ++w) carry = max(carry, s_warp[w]);
  const int32_t prev = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane > 0) carry = max(carry, prev);
  reinterpret_cast<int4*>(s_row)[2 * threadIdx.x] =
      make_int4(max(v[0], carry), max(v[1], carry), max(v[2], carry), max(v[3], carry));
  reinterpret_cast<int4*>(s_row)[2 * threadIdx.x + 1] =
      make_int4(max(v[4], carry), max(v[5], carry), max(v[6], carry), max(v[7], carry));
  __syncthreads();
}

// Binary search of value w in the sorted row v: position or -1.
template <class OffT>
__device__ __forceinline__ int64_t row_find(const OffT* __restrict__ off,
                                            const int32_t* __restrict__ col, int32_t v, int32_t w) {
  int64_t lo = (int64_t)off[v], end = (int64_t)off[v + 1], hi = end;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (col[mid] < w)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < end && col[lo] == w) ? lo : -1;
}

}  // namespace rst
