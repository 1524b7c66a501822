// Bulk-copy streaming loop for the byte-stream kernels (polynomial products, GF(p^k)
// products): per item, two input records (sa and sb bytes) and one output record (so bytes),
// all dense arrays.  A persistent block walks tiles of ITEMS items; thread 0 moves whole
// tiles with the bulk copy engine (cp.async.bulk global -> shared, completion counted on an
// mbarrier; shared -> global as bulk groups), double-buffered in both directions, while all
// threads compute items from shared memory.  Every wait is bounded and reports ERR_TIMEOUT.
//
// Requirements checked by the launcher: base pointers 16-byte aligned; only full tiles here
// (ITEMS * s multiples of 16 by construction); the tail goes to the plain per-thread path.
#pragma once

#include "fpdqt_internal.cuh"

namespace fpd {

static constexpr uint32_t ST_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t st_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void st_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(st_su32(bar)), "r"(count));
}
__device__ __forceinline__ void st_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st_su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool st_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(st_su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool st_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < ST_WAIT_LIMIT; ++i)
    if (st_try(bar, parity)) return true;
  return false;
}
// bulk copy global -> shared, completion on `bar`
__device__ __forceinline__ void st_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   st_su32(dst)),
               "l"(src), "r"(bytes), "r"(st_su32(bar))
               : "memory");
}
// bulk copy shared -> global in the current bulk group
__device__ __forceinline__ void st_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(st_su32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void st_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void st_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void st_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void st_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Op: static constexpr uint32_t IPT (items per thread);
//     __device__ void item(const uint8_t* a, const uint8_t* b, uint8_t* out) for one item
//     (all threads call it IPT times per tile, uniformly).
// Shared layout: [inA 2x][inB 2x][out 2x] tiles, then 2 mbarriers.
template <typename Op>
__device__ void stream_tiles(Op& op, const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                             uint8_t* __restrict__ C, uint64_t ntiles, uint32_t sa, uint32_t sb, uint32_t so,
                             uint8_t* smem, uint32_t* err) {
  constexpr uint32_t ITEMS = 256 * Op::IPT;
  const uint32_t ta = ITEMS * sa, tb = ITEMS * sb, to = ITEMS * so;
  // buffer x of each double pair, by arithmetic (an indexed local array would live in memory)
  auto inA = [&](int x) { return smem + x * ta; };
  auto inB = [&](int x) { return smem + 2 * ta + x * tb; };
  auto out = [&](int x) { return smem + 2 * ta + 2 * tb + x * to; };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * (ta + tb + to));
  __shared__ uint32_t s_abort;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    st_mbar_init(&full[0], 1);
    st_mbar_init(&full[1], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // my tiles: t_i = blockIdx.x + i * gridDim.x
  const uint64_t first = blockIdx.x, stride = gridDim.x;
  const uint64_t mine = first < ntiles ? (ntiles - first + stride - 1) / stride : 0;
  auto issue = [&](uint64_t i, int buf) {
    const uint64_t t = first + i * stride;
    st_expect_tx(&full[buf], ta + tb);
    st_load(inA(buf), A + t * ta, ta, &full[buf]);
    if (tb) st_load(inB(buf), B + t * tb, tb, &full[buf]);
  };
  if (tid == 0) {
    if (mine > 0) issue(0, 0);
    if (mine > 1) issue(1, 1);
  }
  uint64_t i = 0;
  for (; i < mine; ++i) {
    const int buf = (int)(i & 1);
    if (tid == 0) st_wait_read1();          // the store issued from out[buf] two tiles ago has read it
    __syncthreads();
    if (s_abort) break;
    if (!st_wait(&full[buf], (uint32_t)(i >> 1) & 1u)) {
      s_abort = 1;                           // benign race: every writer stores 1
      flag_error(err, ERR_TIMEOUT);
    }
    __syncthreads();
    if (s_abort) break;
#pragma unroll Op::UNROLL
    for (uint32_t j = 0; j < Op::IPT; ++j) {
      const uint32_t it = j * 256 + tid;
      op.item(inA(buf) + it * sa, inB(buf) + it * sb, out(buf) + it * so);
    }
    st_fence_async();                        // generic-proxy writes of out[buf] -> async proxy
    __syncthreads();                         // all threads done with inA/inB[buf], out[buf] written
    if (tid == 0) {
      const uint64_t t = first + i * stride;
      st_store(C + t * to, out(buf), to);
      st_commit();
      if (i + 2 < mine) issue(i + 2, buf);
    }
  }
  if (tid == 0) {
    st_wait_all();                           // every store has completed
    // loads armed but not consumed (only after an abort): let them land before exit
    for (uint64_t k = i; k < mine && k < i + 2; ++k) st_wait(&full[k & 1], (uint32_t)(k >> 1) & 1u);
  }
  __syncthreads();
}

}  // namespace fpd
