// Union-find over int32 vertex ids with compare-and-swap hooking, shared by
// the sampled connectivity strategy and the biconnected-components pass.
// Reads go to L2 (__ldcg): a stale L1 copy of a root pointer would make the
// CAS fail again and again.  Every loop is bounded by n.
#pragma once

#include "common.cuh"

namespace rst {

// Root of x; halves the path on the way (each write replaces a pointer by an
// ancestor, so concurrent finds and hooks stay correct).
__device__ __forceinline__ int32_t uf_find(int32_t* uf, int32_t x, int64_t n, uint32_t* status) {
  for (int64_t it = 0; it <= n; ++it) {
    const int32_t p = __ldcg(&uf[x]);
    if (p == x) return x;
    const int32_t g = __ldcg(&uf[p]);
    if (g != p) uf[x] = g;
    x = g;
  }
  raise_error(status, DERR_WALK_LIMIT);
  return x;
}

// Root of x without writes.  The compression pass uses it: a halving write
// from a concurrent find could otherwise land after a vertex's final write
// of its root and leave it one step short.
__device__ __forceinline__ int32_t uf_root(const int32_t* uf, int32_t x, int64_t n, uint32_t* status) {
  for (int64_t it = 0; it <= n; ++it) {
    const int32_t p = __ldcg(&uf[x]);
    if (p == x) return x;
    x = p;
  }
  raise_error(status, DERR_WALK_LIMIT);
  return x;
}

// Merges the trees of u and v; true iff this call's CAS did the merge.  A
// failed CAS repeats both finds from u and v: the halving writes of every
// retry shorten the paths other links walk (resuming from the roots found
// instead made the biconnected-components link pass 2.5x slower).
__device__ __forceinline__ bool uf_link(int32_t* uf, int32_t u, int32_t v, int64_t n, uint32_t* status) {
  for (int64_t it = 0; it <= n; ++it) {
    const int32_t ru = uf_find(uf, u, n, status), rv = uf_find(uf, v, n, status);
    if (ru == rv) return false;
    const int32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
    if (atomicCAS(&uf[hi], hi, lo) == hi) return true;
  }
  raise_error(status, DERR_ROUND_LIMIT);
  return false;
}

// Points every vertex at its root (no links may run at the same time).
__global__ void k_uf_compress(int64_t n, int32_t* uf, uint32_t* status);

}  // namespace rst
