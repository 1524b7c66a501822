// tcgen05 / TMA / mbarrier helpers shared by the tensor-core matrix kernels (inline PTX for
// sm_103a) and the host-side tensor-map encoder.
#pragma once

#include <mutex>
#include <unordered_map>

#include <cuda.h>
#include <cuda_fp16.h>

#include "fpdqt_internal.cuh"

namespace fpd {

// fp16 bits of a centred residue of p <= 3 ({0,1,2} -> {0,1,-1}) and of a packed pair
// c(v0) + 2^10 c(v1) (|value| <= 1025 < 2^11: exact in fp16).
__device__ __forceinline__ uint32_t h16_centred(uint32_t v) { return v == 0 ? 0u : (v == 1 ? 0x3C00u : 0xBC00u); }
// fp16 bits of the centred residue of v mod p (v - p when 2v > p), exact for p <= 2047.
__device__ __forceinline__ uint32_t h16_centred_p(uint32_t v, uint32_t p) {
  const float c = 2 * v > p ? (float)v - (float)p : (float)v;
  return __half_as_ushort(__float2half_rn(c));
}
// fp16 bits of c(v0) + Q c(v1) for centred residues; exact while |c0| + Q |c1| <= 2048.
__device__ __forceinline__ uint32_t h16_pair_word_p(uint32_t v0, uint32_t v1, uint32_t p, float Q) {
  const float c0 = 2 * v0 > p ? (float)v0 - (float)p : (float)v0;
  const float c1 = 2 * v1 > p ? (float)v1 - (float)p : (float)v1;
  return __half_as_ushort(__float2half_rn(fmaf(Q, c1, c0)));
}
__device__ __forceinline__ uint32_t h16_pair_word(uint32_t v0, uint32_t v1) {
  const float c0 = v0 == 2 ? -1.0f : (float)v0, c1 = v1 == 2 ? -1.0f : (float)v1;
  return __half_as_ushort(__float2half_rn(fmaf(1024.0f, c1, c0)));
}

static constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;             // try_wait polls before giving up
static constexpr uint32_t TC_DRAIN_LIMIT = 1u << 20;            // polls for own in-flight work

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the abort flag set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag,
                                          uint32_t limit = TC_WAIT_LIMIT) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023u) == 1023u && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Drain wait: bounded, does not give up early on the abort flag (own copies / MMAs in flight).
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_DRAIN_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor for a K-major tile with 128-byte swizzle: 8-row core
// groups 1024 bytes apart (stride byte offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  uint64_t a = (su32(p) & 0x3FFFFu) >> 4;
  uint64_t d = a;
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// Shared-memory matrix descriptor for an MN-major tile with 128-byte swizzle: 128-byte rows
// along MN, one row per k; 8-row core groups 1024 bytes apart along K (stride byte offset)
// and 128-element MN blocks `mn_block_bytes` apart (leading byte offset).
__device__ __forceinline__ uint64_t smem_desc_mn_sw128(const void* p, uint32_t mn_block_bytes) {
  uint64_t d = (su32(p) & 0x3FFFFu) >> 4;
  d |= (uint64_t)((mn_block_bytes >> 4) & 0x3FFFu) << 16;  // leading byte offset
  d |= (uint64_t)(1024 >> 4) << 32;                       // stride byte offset
  d |= (uint64_t)1 << 46;                                 // version
  d |= (uint64_t)2 << 61;                                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: fp32 accumulate, A/B type (0 f16, 1 bf16), both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_type, int M, int N) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// kind::f8f6f4 with e4m3 A and B (format code 0), fp32 accumulate; b_mn: B is MN-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N, bool b_mn = false) {
  return (1u << 4) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 columns per thread, no wait (the caller waits with tmem_wait before using v).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D map of a rows x cols row-major matrix of 16-bit (esize 2) or 8-bit (esize 1) elements
// with leading dimension ld elements (ld * esize a multiple of 16, base 16-byte aligned),
// box = box_rows x (128 bytes of elements), 128-byte swizzle; reads past cols or rows return 0.
// A map is a pure function of its arguments, so encoded maps are kept in a process-wide cache
// (a batch that repeats its operands skips the driver call; bounded, cleared when full).
struct MapKey {
  const void* base;
  uint64_t rows, cols, ld;
  uint32_t box_rows, esize;
  bool operator==(const MapKey& o) const {
    return base == o.base && rows == o.rows && cols == o.cols && ld == o.ld && box_rows == o.box_rows &&
           esize == o.esize;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    uint64_t h = (uint64_t)(uintptr_t)k.base * 0x9E3779B97F4A7C15ull;
    for (uint64_t v : {k.rows, k.cols, k.ld, (uint64_t)k.box_rows << 8 | k.esize}) h = (h ^ v) * 0x100000001B3ull;
    return (size_t)h;
  }
};
inline std::mutex& map_cache_mu() {
  static std::mutex m;
  return m;
}
inline std::unordered_map<MapKey, CUtensorMap, MapKeyHash>& map_cache() {
  static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> c;
  return c;
}

inline fp_status make_map_ld(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                             uint32_t box_rows, uint32_t esize) {
  const MapKey key{base, rows, cols, ld, box_rows, esize};
  {
    std::lock_guard<std::mutex> lk(map_cache_mu());
    auto it = map_cache().find(key);
    if (it != map_cache().end()) {
      *map = it->second;
      return FP_OK;
    }
  }
  EncodeTiledFn enc = get_encode();
  FP_CHECK(enc != nullptr, FP_ECUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esize), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                   const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FP_CHECK(r == CUDA_SUCCESS, FP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  std::lock_guard<std::mutex> lk(map_cache_mu());
  if (map_cache().size() >= 65536) map_cache().clear();
  map_cache().emplace(key, *map);
  return FP_OK;
}
inline fp_status make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t kp, uint32_t box_rows,
                          uint32_t esize = 2) {
  return make_map_ld(map, base, rows, kp, kp, box_rows, esize);
}

}  // namespace fpd
