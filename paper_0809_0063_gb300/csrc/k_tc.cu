// Dispatch of the tensor-core matrix products mod p (tcgen05, TMEM accumulators, TMA):
//
//  PLAIN_F8  C = A B mod p, p <= 17, on kind::f8f6f4 with the caller's residue bytes read as
//            e4m3 operands (k_tcg.cu).  A or B whose layout the TMA cannot address directly
//            (base not 16-byte aligned, or a leading dimension not a multiple of 16) is first
//            copied into context scratch with a padded leading dimension.
//  PLAIN_TC  C = A B mod p on kind::f16 with bf16 operands (k_tcp.cu, plain form).
//  RIGHT_TC  right compression (Sec. 7.4) on kind::f16: two centred residues of B per fp16
//            operand word, chunked delayed reduction and REDQ_2 (k_tcp.cu, packed form).
//
// It also holds the self-test of the bounded mbarrier wait that every tensor-core kernel uses.
#include <algorithm>

#include "fpdqt_internal.cuh"
#include "tc_ptx.cuh"

namespace fpd {

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing will complete,
// gives up after `polls` polls and reports ERR_TIMEOUT through the context's flag -- the
// same path the tensor-core kernels take when a TMA or MMA completion never arrives.
__global__ void k_selftest_wait(uint32_t polls, uint32_t* err) {
  __shared__ uint64_t bar;
  __shared__ uint32_t abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(&bar, 0, &abort_flag, polls)) flag_error(err, ERR_TIMEOUT);
    mbar_arrive(&bar);   // complete the phase so the barrier is left in a finished state
  }
  __syncthreads();
}

// The caller holds the context lock.
fp_status launch_mm_tc(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                       int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st) {
  fp_status s = mm_bound_check(p, k, algo);
  if (s != FP_OK) return s;
  if (algo == FP_MM_PLAIN_TC || algo == FP_MM_RIGHT_TC) {
    const fp_mm_problem x = {p, m, n, k, A, lda, B, ldb, C, ldc};
    return launch_mm_t16_direct(ctx, x, algo == FP_MM_RIGHT_TC, st);
  }
  // PLAIN_F8
  fp_mm_problem x = {p, m, n, k, A, lda, B, ldb, C, ldc};
  if (!f8_direct_ok(p, k, A, lda, B, ldb)) {
    // pad copies (no arithmetic): rows of A and B at leading dimensions rounded up to 16
    const size_t lda2 = ((size_t)k + 15) / 16 * 16, ldb2 = ((size_t)n + 15) / 16 * 16;
    const size_t abytes = ((size_t)m * lda2 + 1023) & ~(size_t)1023, bbytes = (size_t)k * ldb2;
    s = ensure_scratch(ctx, abytes + bbytes + 1024, 0, st);
    if (s != FP_OK) return s;
    uint8_t* A2 = (uint8_t*)ctx->scratch;
    uint8_t* B2 = A2 + abytes;
    FP_CUDA(cudaMemcpy2DAsync(A2, lda2, A, (size_t)lda, (size_t)k, (size_t)m, cudaMemcpyDeviceToDevice, st));
    FP_CUDA(cudaMemcpy2DAsync(B2, ldb2, B, (size_t)ldb, (size_t)n, (size_t)k, cudaMemcpyDeviceToDevice, st));
    x.A = A2;
    x.lda = (int)lda2;
    x.B = B2;
    x.ldb = (int)ldb2;
  }
  return launch_mm_f8_direct(ctx, x, st);
}

}  // namespace fpd

extern "C" fp_status fp_selftest_bounded_wait(fp_ctx ctx, uint32_t polls, void* stream) {
  using namespace fpd;
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_selftest_bounded_wait: ctx is NULL");
  FP_CHECK(polls >= 1 && polls <= (1u << 22), FP_EINVAL, "fp_selftest_bounded_wait: polls in [1, 2^22]");
  cudaStream_t st = as_stream(stream);
  FP_LAUNCH(ctx, "k_selftest_wait", st, k_selftest_wait<<<1, 32, 0, st>>>(polls, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}
