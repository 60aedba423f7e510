// Path-reversal RST (Section III-C).
#include "pipeline.cuh"
#include "strategies.cuh"

namespace rst {

rst_status run_prrst(const void* off, int offsets_bits, const int32_t* cols, int64_t n, int64_t m,
                     int32_t root, int32_t* parent, cudaStream_t s) {
  (void)off; (void)offsets_bits; (void)cols; (void)n; (void)m; (void)root; (void)parent; (void)s;
  return RST_ERR_UNSUPPORTED;
}

rst_strategy select_strategy_host(const void* off, int offsets_bits, const int32_t* cols, int64_t n,
                                  int64_t m, int32_t root, cudaStream_t s) {
  (void)off; (void)offsets_bits; (void)cols; (void)n; (void)m; (void)root; (void)s;
  return RST_CC_EULER;
}

}  // namespace rst
