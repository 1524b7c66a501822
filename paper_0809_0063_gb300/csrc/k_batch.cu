// Uneven batches in one persistent launch: placeholder until the work-queue kernel lands.
#include "fpdqt_internal.cuh"

extern "C" fp_status fp_batch_run(fp_ctx ctx, const fp_instance* instances, size_t count, void* stream) {
  (void)ctx; (void)instances; (void)count; (void)stream;
  fpd::set_error("fp_batch_run: not built");
  return FP_EUNSUPPORTED;
}
