// Strategy drivers behind rst_build / rst_verify (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace rst {

// Level-synchronous, direction-optimising BFS (Section III-A).  level_out
// (nullable) receives each vertex's distance from its component's source.
rst_status run_bfs(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                   int32_t root, int32_t* parent, int32_t* level_out, cudaStream_t s);

// The same search with the level loop on the device: one kernel per level
// inside a CUDA-graph while node, or (persistent) one cooperative launch whose
// blocks meet at a bounded grid barrier after each level.  No host
// synchronisation per level.
rst_status run_bfs_device(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                          int32_t root, int32_t* parent, int32_t* level_out, cudaStream_t s,
                          bool persistent);
void destroy_bfs_graphs();

// A bounded BFS from the root (the selector's probe): frontier sizes of the
// first levels, vertices reached, whether the search finished.
struct BfsProbe {
  static constexpr int kMax = 64;
  int max_levels = 8;
  int levels = 0;
  bool finished = false;
  long long reached = 0;
  long long last_frontier = 0;
  long long frontier[kMax] = {0};
};
rst_status bfs_probe_in(Arena& ar, const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                        int32_t root, int32_t* parent_scratch, BfsProbe* probe, cudaStream_t s);
void set_bfs_max_levels(long long v);
long long get_bfs_max_levels();

// BFS from several sources at once (the roots of a disjoint union), with
// buffers taken from the caller's arena (bfs_workspace_bytes(n) of room).
size_t bfs_workspace_bytes(int64_t n);
rst_status bfs_multi_in(Arena& ar, const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                        const int32_t* seeds, int64_t nseeds, int32_t* parent, cudaStream_t s);

// Path-reversal RST (Section III-C).
rst_status run_prrst(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                     int32_t root, int32_t* parent, cudaStream_t s);

// Exact verdict of a parent array.
// Blocks and cut vertices (bcc.cu).
template <class OffT>
size_t bcc_workspace_bytes(int64_t n, int64_t A);
template <class OffT>
rst_status bcc_run(Arena& ar, const OffT* off, const int32_t* col, int64_t n, int64_t A, uint32_t* label,
                   uint8_t* cut, int64_t* nblocks, cudaStream_t s);
// Depth of every vertex of a rooted forest (depth.cu); the workspace must
// hold depth_workspace_bytes(n).
size_t depth_workspace_bytes(int64_t n);
rst_status tree_depth(const int32_t* parent, int64_t n, int32_t* depth_out, int64_t* max_out,
                      cudaStream_t s);
// PR-RST rounds started from the rooted forest in `parent` over k inserted
// edges (uv pairs); the result replaces `parent` (prrst.cu).
rst_status run_prrst_insert(int64_t n, int32_t* parent, const int32_t* uv, int64_t k, int32_t root,
                            bool canonical, cudaStream_t s);
rst_status run_verify(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                      int32_t root, const int32_t* parent, int32_t* verdict_out, cudaStream_t s);

// Release the device copies of the selector model (rst_shutdown).
void release_selector();

// Strategy for RST_AUTO.
rst_strategy select_strategy_host(const void* off, int offsets_bits, const int32_t* cols, int64_t n,
                                  int64_t m, int32_t root, cudaStream_t s);

}  // namespace rst
