// tcgen05 (5th-generation tensor core) matrix products: placeholder until the kernels land.
#include "fpdqt_internal.cuh"

namespace fpd {
fp_status launch_mm_tc(fp_ctx, uint32_t, int, int, int, const uint8_t*, int, const uint8_t*, int, uint8_t*, int,
                       int algo, cudaStream_t) {
  set_error("fp_matmul: tcgen05 algorithm %d not built", algo);
  return FP_EUNSUPPORTED;
}
}  // namespace fpd
