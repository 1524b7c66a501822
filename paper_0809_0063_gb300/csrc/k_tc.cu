// Matrix products mod p on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA).
//
//  PLAIN_TC  C = A B mod p with A, B converted to bf16 (entries < p <= 256 are exact), one
//            tcgen05.mma kind::f16 contraction with fp32 accumulation in TMEM (exact while the
//            integer sums stay below 2^24, i.e. k (p-1)^2 < 2^24), then mod p in the epilogue.
//  RIGHT_TC  right compression (Sec. 7.4) on the tensor cores: B's columns are packed two per
//            fp16 operand at Q = 2^10 with centred residues (p <= 3: {-1, 0, 1}), so one MMA
//            column carries two residues of C.  Each chunk of 448 inner-dimension steps keeps
//            every digit in (-512, 512) (Eq. lower per chunk, centred); its TMEM accumulator is
//            drained by the epilogue warps into a 32-bit word R = D0 + 2^16 D1 while the MMA
//            warp fills the other TMEM buffer (delayed reduction, Sec. 2.2).  At the end an
//            offset makes both digits non-negative and REDQ_2 (Algorithm 2) recovers them mod p.
//  PLAIN_F8  C = A B mod p on kind::f8f6f4 with e4m3 operands, p <= 17.  Residues 0..16 read
//            as e4m3 bit patterns are exactly r 2^-9 (codes 0..7 subnormal, 8..15 the first
//            binade, 16 = 2^-5), so when A and B are 16-byte aligned with leading dimensions
//            a multiple of 16 the persistent grouped kernel streams the caller's bytes
//            directly (k_tcg.cu).  Other layouts are converted here to e4m3 of the integer
//            values (K-major, zero padded) for the kernel below.
//
// Kernel roles (one CTA = one 128 x 256 output tile of words, 1 CTA per SM):
//   warp 0       TMA producer: A tile 128 x 64 and B tile 256 x 64 (bf16/fp16, 128-byte
//                swizzle) per stage into a 4-stage shared-memory ring (mbarrier full/empty),
//   warp 1       TMEM allocation and the single MMA-issuing thread,
//   warps 2..9   epilogue: tcgen05.ld of the accumulator, decode / mod p, stores to C.
// Every mbarrier wait is bounded; a wait that gives up sets the context's error flag
// (ERR_TIMEOUT), lets the other roles drain, frees TMEM and returns.
#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fpdqt_internal.cuh"
#include "tc_ptx.cuh"

namespace fpd {

static constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 4;
static constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;            // 16 KB
static constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;            // 32 KB
static constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;  // 48 KB
static constexpr int TC_THREADS = 320;                          // 10 warps
static constexpr int TC_CHUNK_KT = 7;                           // 448 inner steps per packed chunk

// ---------------------------------------------------------------- operand conversion

// bf16 bits of a residue v <= 255: the float 2^23 + v has v in its low mantissa bits, so
// subtracting 2^23 gives float(v) exactly; its top 16 bits are the bf16 (exact, 8 bits).
__device__ __forceinline__ uint32_t bf16_pair(uint32_t v0, uint32_t v1) {
  const float f0 = __uint_as_float(0x4B000000u | v0) - 8388608.0f;
  const float f1 = __uint_as_float(0x4B000000u | v1) - 8388608.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}
// fp16 bits of a centred residue of p = 3 ({0,1,2} -> {0,1,-1}) and of a packed pair
// c(v0) + 2^10 c(v1): 9 possible values, looked up from (v0, v1).
__device__ __forceinline__ uint32_t h16_centred(uint32_t v) { return v == 0 ? 0u : (v == 1 ? 0x3C00u : 0xBC00u); }
__device__ __forceinline__ uint32_t h16_pair_word(uint32_t v0, uint32_t v1) {
  const float c0 = v0 == 2 ? -1.0f : (float)v0, c1 = v1 == 2 ? -1.0f : (float)v1;
  return __half_as_ushort(__float2half_rn(fmaf(1024.0f, c1, c0)));
}

// A16[r][c] (m x kp, zero padded) = 16-bit form of A[r][c]; one thread per 16 columns.
// mode 0 bf16, mode 1 fp16 of the centred residue (p <= 3).
__global__ void __launch_bounds__(256) k_tc_convert_a(const uint8_t* __restrict__ A, int lda, uint16_t* __restrict__ dst,
                                                      int m, int k, int kp, int mode, uint32_t p, uint32_t* err) {
  const int chunks = kp >> 4;
  uint32_t bad = 0;
  const bool vec = (((uintptr_t)A) & 15u) == 0 && (lda & 15) == 0;
  for (int r = blockIdx.x; r < m; r += gridDim.x)
    for (int ch = threadIdx.x; ch < chunks; ch += blockDim.x) {
      const int c0 = ch * 16;
      uint32_t w[4];
      const uint8_t* src = A + (size_t)r * lda + c0;
      if (vec && c0 + 16 <= k) {
        uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t t = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) t |= (uint32_t)(c0 + 4 * q + j < k ? src[4 * q + j] : 0) << (8 * j);
          w[q] = t;
        }
      }
      const uint32_t pp = 0x01010101u * p;
      bad |= __vcmpgeu4(w[0], pp) | __vcmpgeu4(w[1], pp) | __vcmpgeu4(w[2], pp) | __vcmpgeu4(w[3], pp);
      uint32_t o[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t x = w[q];
        const uint32_t b0 = x & 0xffu, b1 = (x >> 8) & 0xffu, b2 = (x >> 16) & 0xffu, b3 = x >> 24;
        if (mode == 0) {
          o[2 * q] = bf16_pair(b0, b1);
          o[2 * q + 1] = bf16_pair(b2, b3);
        } else {
          o[2 * q] = h16_centred(b0) | (h16_centred(b1) << 16);
          o[2 * q + 1] = h16_centred(b2) | (h16_centred(b3) << 16);
        }
      }
      uint4* d = reinterpret_cast<uint4*>(dst + (size_t)r * kp + c0);
      d[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// B16 (nw x kp, zero padded) from B (k x n): a 64 (k) x 64 (n) tile of B per block is staged
// in shared memory as 32-bit words; each thread transposes one 4 x 4 byte block in registers
// (__byte_perm) and writes 4 k-values for each of its 4 columns.  mode 0: bf16 of B[c][w]
// (nw = n); mode 2: fp16 of the centred pair B[c][2w] + 2^10 B[c][2w+1] (nw = ceil(n/2)).
__global__ void __launch_bounds__(256) k_tc_convert_b(const uint8_t* __restrict__ B, int ldb, uint16_t* __restrict__ dst,
                                                      int k, int n, int nw, int kp, int mode, uint32_t p, uint32_t* err) {
  __shared__ uint32_t tile[64][17];                 // 64 rows (k) x 64 bytes (n), row stride 17 words
  const int c0 = blockIdx.x * 64;                   // k offset
  const int n0 = blockIdx.y * 64;                   // B column offset
  const int t = threadIdx.x;
  uint32_t bad = 0;
  {
    const int rr = t >> 2, cc = (t & 3) * 16;       // 64 rows x 4 chunks of 16 columns
    const int kr = c0 + rr, col = n0 + cc;
    uint32_t w[4];
    const uint8_t* src = B + (size_t)kr * ldb + col;
    if (kr < k && col + 16 <= n && (((uintptr_t)src) & 15u) == 0) {
      uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
      w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) v |= (uint32_t)((kr < k && col + 4 * q + j < n) ? src[4 * q + j] : 0) << (8 * j);
        w[q] = v;
      }
    }
    const uint32_t pp = 0x01010101u * p;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bad |= __vcmpgeu4(w[q], pp);
      tile[rr][(cc >> 2) + q] = w[q];
    }
  }
  __syncthreads();
  const int bk = t & 15, bn = t >> 4;               // 4 x 4 block: k rows 4bk.., columns 4bn..
  const uint32_t r0 = tile[4 * bk][bn], r1 = tile[4 * bk + 1][bn], r2 = tile[4 * bk + 2][bn], r3 = tile[4 * bk + 3][bn];
  // transpose: column j gathers byte j of r0..r3 (k order)
  const uint32_t lo01 = __byte_perm(r0, r1, 0x5140), hi01 = __byte_perm(r0, r1, 0x7362);
  const uint32_t lo23 = __byte_perm(r2, r3, 0x5140), hi23 = __byte_perm(r2, r3, 0x7362);
  uint32_t col[4];
  col[0] = __byte_perm(lo01, lo23, 0x5410);         // bytes: r0[0] r1[0] r2[0] r3[0]
  col[1] = __byte_perm(lo01, lo23, 0x7632);         // r0[1] r1[1] r2[1] r3[1]
  col[2] = __byte_perm(hi01, hi23, 0x5410);
  col[3] = __byte_perm(hi01, hi23, 0x7632);
  const int kk = c0 + 4 * bk;                      // < kp: the grid covers kp / 64 tiles
  if (mode == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int w = n0 + 4 * bn + j;
      if (w >= nw) break;
      const uint32_t x = col[j];
      uint2 o = make_uint2(bf16_pair(x & 0xffu, (x >> 8) & 0xffu), bf16_pair((x >> 16) & 0xffu, x >> 24));
      *reinterpret_cast<uint2*>(dst + (size_t)w * kp + kk) = o;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int w = n0 / 2 + 2 * bn + j;
      if (w >= nw) break;
      const uint32_t x0 = col[2 * j], x1 = col[2 * j + 1];   // columns 2w and 2w+1
      uint32_t h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) h[q] = h16_pair_word((x0 >> (8 * q)) & 0xffu, (x1 >> (8 * q)) & 0xffu);
      *reinterpret_cast<uint2*>(dst + (size_t)w * kp + kk) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    }
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// e4m3 bits of a residue v <= 16 (exact): exponent floor(log2 v) + 7, three mantissa bits.
__device__ __forceinline__ uint32_t e4m3_of(uint32_t v) {
  if (v == 0) return 0u;
  const uint32_t e = 31u - __clz(v);
  return ((e + 7u) << 3) | (((v << 3) >> e) & 7u);
}
__device__ __forceinline__ uint32_t e4m3_word(uint32_t x) {   // four bytes at once
  return e4m3_of(x & 0xffu) | (e4m3_of((x >> 8) & 0xffu) << 8) | (e4m3_of((x >> 16) & 0xffu) << 16) |
         (e4m3_of(x >> 24) << 24);
}

// A8[r][c] (m x kp, zero padded) = e4m3 of A[r][c]; one thread per 16 columns.
__global__ void __launch_bounds__(256) k_tc_convert_a8(const uint8_t* __restrict__ A, int lda, uint8_t* __restrict__ dst,
                                                       int m, int k, int kp, uint32_t p, uint32_t* err) {
  const int chunks = kp >> 4;
  uint32_t bad = 0;
  const bool vec = (((uintptr_t)A) & 15u) == 0 && (lda & 15) == 0;
  for (int r = blockIdx.x; r < m; r += gridDim.x)
    for (int ch = threadIdx.x; ch < chunks; ch += blockDim.x) {
      const int c0 = ch * 16;
      uint32_t w[4];
      const uint8_t* src = A + (size_t)r * lda + c0;
      if (vec && c0 + 16 <= k) {
        uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t t = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) t |= (uint32_t)(c0 + 4 * q + j < k ? src[4 * q + j] : 0) << (8 * j);
          w[q] = t;
        }
      }
      const uint32_t pp = 0x01010101u * p;
      bad |= __vcmpgeu4(w[0], pp) | __vcmpgeu4(w[1], pp) | __vcmpgeu4(w[2], pp) | __vcmpgeu4(w[3], pp);
      *reinterpret_cast<uint4*>(dst + (size_t)r * kp + c0) =
          make_uint4(e4m3_word(w[0]), e4m3_word(w[1]), e4m3_word(w[2]), e4m3_word(w[3]));
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// B8 (n x kp, zero padded) = e4m3 of B transposed: 64 (k) x 64 (n) tiles, 4 x 4 byte blocks
// transposed in registers, 4 k-values per column written as one 32-bit store.
__global__ void __launch_bounds__(256) k_tc_convert_b8(const uint8_t* __restrict__ B, int ldb, uint8_t* __restrict__ dst,
                                                       int k, int n, int kp, uint32_t p, uint32_t* err) {
  __shared__ uint32_t tile[64][17];
  const int c0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int t = threadIdx.x;
  uint32_t bad = 0;
  {
    const int rr = t >> 2, cc = (t & 3) * 16;
    const int kr = c0 + rr, col = n0 + cc;
    uint32_t w[4];
    const uint8_t* src = B + (size_t)kr * ldb + col;
    if (kr < k && col + 16 <= n && (((uintptr_t)src) & 15u) == 0) {
      uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
      w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) v |= (uint32_t)((kr < k && col + 4 * q + j < n) ? src[4 * q + j] : 0) << (8 * j);
        w[q] = v;
      }
    }
    const uint32_t pp = 0x01010101u * p;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bad |= __vcmpgeu4(w[q], pp);
      tile[rr][(cc >> 2) + q] = w[q];
    }
  }
  __syncthreads();
  const int bk = t & 15, bn = t >> 4;
  const uint32_t r0 = tile[4 * bk][bn], r1 = tile[4 * bk + 1][bn], r2 = tile[4 * bk + 2][bn], r3 = tile[4 * bk + 3][bn];
  const uint32_t lo01 = __byte_perm(r0, r1, 0x5140), hi01 = __byte_perm(r0, r1, 0x7362);
  const uint32_t lo23 = __byte_perm(r2, r3, 0x5140), hi23 = __byte_perm(r2, r3, 0x7362);
  uint32_t col[4];
  col[0] = __byte_perm(lo01, lo23, 0x5410);
  col[1] = __byte_perm(lo01, lo23, 0x7632);
  col[2] = __byte_perm(hi01, hi23, 0x5410);
  col[3] = __byte_perm(hi01, hi23, 0x7632);
  const int kk = c0 + 4 * bk;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int w = n0 + 4 * bn + j;
    if (w >= n) break;
    *reinterpret_cast<uint32_t*>(dst + (size_t)w * kp + kk) = e4m3_word(col[j]);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// ---------------------------------------------------------------- the GEMM kernel

// MODE 0: bf16 plain, 1: fp16 packed (two centred residues per word), 2: e4m3 plain from
// converted operands.
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_mm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, uint8_t* __restrict__ C,
            int ldc, uint32_t* __restrict__ RW, int m, int n, int nw, int ktiles, RedqParams P, uint32_t koffset,
            uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* tfull = empty + TC_STAGES;   // [2] accumulator ready
  uint64_t* tempty = tfull + 2;          // [2] accumulator drained
  uint64_t* drainb = tempty + 2;         // MMA completion on the abort path
  uint64_t* doneb = drainb + 1;          // every epilogue warp finished with TMEM
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(doneb + 1);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  __shared__ uint8_t ptab[1024];

  constexpr bool PACKED = MODE == 1;
  constexpr int KT_ELEMS = MODE == 2 ? 128 : 64;   // elements per 128-byte k-tile row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  constexpr uint32_t TMEM_COLS = PACKED ? 512 : 256;
  const int nchunks = PACKED ? (ktiles + TC_CHUNK_KT - 1) / TC_CHUNK_KT : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);      // one arrival per epilogue warp
    }
    mbar_init(drainb, 1);
    mbar_init(doneb, 8);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fill_pair_table(ptab, P);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int armed = 0;
      for (int kt = 0; kt < ktiles && !*abort_flag; ++kt) {
        const int s = kt % TC_STAGES;
        const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) break;
        uint8_t* sa = smem + s * TC_STAGE_BYTES;
        uint8_t* sb = sa + TC_A_BYTES;
        mbar_expect_tx(&full[s], TC_STAGE_BYTES);
        tma_load_2d(sa, &tmA, kt * KT_ELEMS, m0, &full[s]);
        tma_load_2d(sb, &tmB, kt * KT_ELEMS, n0, &full[s]);
        armed = kt + 1;
      }
      // every armed stage must have landed before the CTA may exit (its shared memory is reused)
      for (int kt = (armed > TC_STAGES ? armed - TC_STAGES : 0); kt < armed; ++kt)
        mbar_drain(&full[kt % TC_STAGES], (uint32_t)(kt / TC_STAGES) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc =
          MODE == 2 ? idesc_e4m3(TC_BM, TC_BN) : idesc_f16(PACKED ? 0u : 1u, TC_BM, TC_BN);
      int kt = 0;
      for (int c = 0; c < nchunks && !*abort_flag; ++c) {
        const int buf = c & 1;
        const uint32_t dtm = tmem + (uint32_t)(buf * 256);
        if (c >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((c - 2) >> 1) & 1u, abort_flag)) break;
        tc_fence_after();
        const int kend = PACKED ? min(ktiles, kt + TC_CHUNK_KT) : ktiles;
        bool first = true;
        for (; kt < kend; ++kt) {
          const int s = kt % TC_STAGES;
          if (!mbar_wait(&full[s], (uint32_t)(kt / TC_STAGES) & 1u, abort_flag)) break;
          tc_fence_after();
          const uint8_t* sa = smem + s * TC_STAGE_BYTES;
          const uint8_t* sb = sa + TC_A_BYTES;
          const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_sw128(sb);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // advance 32 bytes along K inside the swizzled 128-byte rows (16 x 16-bit or 32 x fp8)
            if (MODE == 2) mma_f8(dtm, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, first ? 0u : 1u);
            else mma_f16(dtm, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, first ? 0u : 1u);
            first = false;
          }
          mma_commit(&empty[s]);    // stage s free once these MMAs have read it
        }
        mma_commit(&tfull[buf]);    // accumulator buffer ready once all MMAs completed
      }
      if (*abort_flag) {            // wait for every MMA issued so far before TMEM is freed
        mma_commit(drainb);
        mbar_drain(drainb, 0);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2..9)
    Corrector corr;
    corr.init(P, ptab);
    const int q = warp & 3;                      // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;            // column half (0: 0..127, 1: 128..255)
    const int row = m0 + q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    if (!PACKED) {
      bool ok = mbar_wait(&tfull[0], 0, abort_flag);
      tc_fence_after();
      for (int cb = 0; cb < 4 && ok; ++cb) {
        const int col0 = half * 128 + cb * 32;
        uint32_t v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)col0, v);
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          uint32_t w = 0;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            uint32_t x = __float2uint_rn(__uint_as_float(v[j + t]));
            w |= modp32(x, P.dv, P.p) << (8 * t);
          }
          packed[j >> 2] = w;
        }
        const int c0 = n0 + col0;
        if (row < m) {
          uint8_t* dst = C + (size_t)row * ldc + c0;
          if (c0 + 32 <= n && ((((uintptr_t)dst) & 15u) == 0)) {
            reinterpret_cast<uint4*>(dst)[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            reinterpret_cast<uint4*>(dst)[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
          } else {
            for (int j = 0; j < 32 && c0 + j < n; ++j) dst[j] = (uint8_t)(packed[j >> 2] >> (8 * (j & 3)));
          }
        }
      }
    } else {
      // R = D0 + 2^16 D1 per word of this thread's 128 columns, accumulated over the chunks
      uint32_t R[128];   // unsigned: wraps modulo 2^32 (the magic offsets cancel at the end)
#pragma unroll
      for (int j = 0; j < 128; ++j) R[j] = 0;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (ok) ok = mbar_wait(&tfull[buf], (uint32_t)(c >> 1) & 1u, abort_flag);
        tc_fence_after();
        if (ok) {
          // 8 blocks of 16 columns, loads double-buffered so each block's TMEM latency overlaps
          // the previous block's arithmetic.  Chunk word v = d0 + 2^10 d1, |d0|, |d1| <= 448:
          // adding 1.5 2^23 makes the float's bits 0x4B400000 + v exactly (|v| < 2^22), so
          // y - 0x4B400000 = v without a conversion instruction; d1 = round(v / 2^10).
          const uint32_t base = tmem + lane_base + (uint32_t)(buf * 256 + half * 128);
          uint32_t va[16], vb[16];
          tmem_ld16_nowait(base, va);
          tmem_wait();
#pragma unroll
          for (int blk = 0; blk < 8; ++blk) {
            if (blk + 1 < 8) {
              if (blk & 1) tmem_ld16_nowait(base + (uint32_t)((blk + 1) * 16), va);
              else tmem_ld16_nowait(base + (uint32_t)((blk + 1) * 16), vb);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const uint32_t raw = (blk & 1) ? vb[j] : va[j];
              const int32_t y = __float_as_int(__uint_as_float(raw) + 12582912.0f);
              const int32_t d1 = (y - (0x4B400000 - 512)) >> 10;
              R[blk * 16 + j] += (uint32_t)y + (uint32_t)(d1 * (65536 - 1024));
            }
            tmem_wait();
          }
        }
        tc_fence_before();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      // The word CC = D0 + 2^16 D1 of this thread's row and 128 columns goes to global memory
      // with both digits made non-negative by the offset koffset (>= every |digit|) and the
      // per-chunk conversion constant removed; a separate pass applies REDQ (Eq. LeftComp:
      // CC = A x CB, then REDQ(CC)).
      const uint32_t fix = koffset * 65537u - (uint32_t)nchunks * 0x4B400000u;
      const int cw0 = n0 + half * 128;
      if (ok && row < m) {
        uint32_t* dst = RW + (size_t)row * nw + cw0;
        if (cw0 + 128 <= nw && (nw & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 128; j += 4)
            *reinterpret_cast<uint4*>(dst + j) = make_uint4(R[j] + fix, R[j + 1] + fix, R[j + 2] + fix, R[j + 3] + fix);
        } else {
#pragma unroll
          for (int j = 0; j < 128; ++j)
            if (cw0 + j < nw) dst[j] = R[j] + fix;
        }
      }
    }
    __syncwarp();
    tc_fence_before();
    if (lane == 0) mbar_arrive(doneb);
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) flag_error(err, ERR_TIMEOUT);
  if (warp == 1) {
    // TMEM is freed only after every epilogue warp has signalled that it is done with it
    if (lane == 0) mbar_drain(doneb, 0);
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// REDQ_2 of the right-compressed product's words (q = 2^16, digits offset by koffset):
// C[r][2w + t] = (digit_t(RW[r][w]) - koffset) mod p.  One thread per 8 words (16 residues,
// one 16-byte store); whole warps iterate so the shuffle-table lookups see 32 lanes.
__global__ void __launch_bounds__(256) k_tc_redq(const uint32_t* __restrict__ RW, uint8_t* __restrict__ C, int ldc,
                                                 int m, int n, int nw, RedqParams P, uint32_t offset_mod_p) {
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector corr;
  corr.init(P, ptab);
  const int groups = (nw + 7) / 8;
  const int gblocks = (groups + (int)blockDim.x - 1) / (int)blockDim.x;   // blocks of threads per row
#pragma unroll 2
  for (int rb = blockIdx.x; rb < m * gblocks; rb += gridDim.x) {
    const int r = rb / gblocks, g = (rb - r * gblocks) * (int)blockDim.x + (int)threadIdx.x;
    const bool own = g < groups;
    const uint32_t* src = RW + (size_t)r * nw + g * 8;
    uint32_t w[8];
    if (own && g * 8 + 8 <= nw && (nw & 3) == 0) {
      uint4 a = *reinterpret_cast<const uint4*>(src);
      uint4 b = *reinterpret_cast<const uint4*>(src + 4);
      w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = (own && g * 8 + j < nw) ? src[j] : 0u;
    }
    uint32_t o[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t mu0, mu1;
      redq2_u32(w[j], P, corr, mu0, mu1);
      uint32_t r0 = mu0 + P.p - offset_mod_p, r1 = mu1 + P.p - offset_mod_p;
      r0 = r0 >= P.p ? r0 - P.p : r0;
      r1 = r1 >= P.p ? r1 - P.p : r1;
      o[j >> 1] |= (r0 | (r1 << 8)) << (16 * (j & 1));
    }
    if (own) {
      const int c0 = 16 * g;
      uint8_t* dst = C + (size_t)r * ldc + c0;
      if (c0 + 16 <= n && ((((uintptr_t)dst) & 15u) == 0)) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(o[0], o[1], o[2], o[3]);
      } else {
        for (int b = 0; b < 16 && c0 + b < n; ++b) dst[b] = (uint8_t)(o[b >> 2] >> (8 * (b & 3)));
      }
    }
  }
}

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


fp_status launch_mm_tc(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                       int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st) {
  const bool packed = algo == FP_MM_RIGHT_TC;
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  if (algo == FP_MM_PLAIN_F8) {
    // residues <= 16 are exact in e4m3; fp32 accumulation exact below 2^24
    FP_CHECK(p <= 17, FP_EBOUND, "PLAIN_F8 needs p <= 17 (p=%u)", p);
    FP_CHECK((uint64_t)k * pp < (1ull << 24), FP_EBOUND, "PLAIN_F8 needs k (p-1)^2 < 2^24");
    const int kp8 = (k + 127) / 128 * 128;
    const size_t smem8 = 1024 + TC_STAGES * TC_STAGE_BYTES + 256;
    dim3 grid8((n + TC_BN - 1) / TC_BN, (m + TC_BM - 1) / TC_BM);
    RedqParams P8 = make_redq(p, 16, 1);
    if (f8_direct_ok(p, k, A, lda, B, ldb)) {
      // the caller's bytes are the e4m3 operands (r 2^-9): the persistent grouped kernel
      const fp_mm_problem x = {p, m, n, k, A, lda, B, ldb, C, ldc};
      return launch_mm_f8_direct(ctx, x, st);
    }
    const size_t ab = ((size_t)m * kp8 + 1023) & ~(size_t)1023, bb = ((size_t)n * kp8 + 1023) & ~(size_t)1023;
    fp_status s8 = ensure_scratch(ctx, ab + bb + 1024);
    if (s8 != FP_OK) return s8;
    uint8_t* A8 = (uint8_t*)ctx->scratch;
    uint8_t* B8 = A8 + ab;
    const int g1 = std::min(m, ctx->num_sms * 16);
    FP_LAUNCH(ctx, "k_tc_convert_a", st, k_tc_convert_a8<<<g1, 256, 0, st>>>(A, lda, A8, m, k, kp8, p, ctx->d_err));
    dim3 gb8(kp8 / 64, (n + 63) / 64);
    FP_LAUNCH(ctx, "k_tc_convert_b", st, k_tc_convert_b8<<<gb8, 256, 0, st>>>(B, ldb, B8, k, n, kp8, p, ctx->d_err));
    FP_CUDA(cudaGetLastError());
    CUtensorMap ma8, mb8;
    s8 = make_map(&ma8, A8, (uint64_t)m, (uint64_t)kp8, TC_BM, 1);
    if (s8 != FP_OK) return s8;
    s8 = make_map(&mb8, B8, (uint64_t)n, (uint64_t)kp8, TC_BN, 1);
    if (s8 != FP_OK) return s8;
    FP_CUDA(cudaFuncSetAttribute(k_mm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8));
    FP_LAUNCH(ctx, "k_mm_tc", st,
              k_mm_tc<2><<<grid8, TC_THREADS, smem8, st>>>(ma8, mb8, C, ldc, nullptr, m, n, n, kp8 / 128, P8, 0,
                                                        ctx->d_err));
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  if (packed) {
    FP_CHECK(p <= 3, FP_EBOUND, "RIGHT_TC needs p <= 3 (p=%u)", p);
    FP_CHECK(k <= 32767, FP_EBOUND, "RIGHT_TC needs k <= 32767");
  } else {
    FP_CHECK((uint64_t)k * pp < (1ull << 24), FP_EBOUND, "PLAIN_TC needs k (p-1)^2 < 2^24");
  }
  const int kp = (k + TC_BK - 1) / TC_BK * TC_BK;
  const int nw = packed ? (n + 1) / 2 : n;
  const size_t abytes = ((size_t)m * kp * 2 + 1023) & ~(size_t)1023, bbytes = ((size_t)nw * kp * 2 + 1023) & ~(size_t)1023;
  const size_t wbytes = packed ? (size_t)m * nw * 4 : 0;
  fp_status s = ensure_scratch(ctx, abytes + bbytes + wbytes + 1024);
  if (s != FP_OK) return s;
  uint16_t* A16 = (uint16_t*)ctx->scratch;
  uint16_t* B16 = (uint16_t*)((uint8_t*)ctx->scratch + abytes);
  uint32_t* RW = (uint32_t*)((uint8_t*)ctx->scratch + abytes + bbytes);
  {
    const int g1 = std::min(m, ctx->num_sms * 16);
    FP_LAUNCH(ctx, "k_tc_convert_a", st,
              k_tc_convert_a<<<g1, 256, 0, st>>>(A, lda, A16, m, k, kp, packed ? 1 : 0, p, ctx->d_err));
    dim3 gb(kp / 64, (n + 63) / 64);
    FP_LAUNCH(ctx, "k_tc_convert_b", st,
              k_tc_convert_b<<<gb, 256, 0, st>>>(B, ldb, B16, k, n, nw, kp, packed ? 2 : 0, p, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  CUtensorMap ma, mb;
  s = make_map(&ma, A16, (uint64_t)m, (uint64_t)kp, TC_BM);
  if (s != FP_OK) return s;
  s = make_map(&mb, B16, (uint64_t)nw, (uint64_t)kp, TC_BN);
  if (s != FP_OK) return s;
  const size_t smem = 1024 + TC_STAGES * TC_STAGE_BYTES + 256;
  dim3 grid((nw + TC_BN - 1) / TC_BN, (m + TC_BM - 1) / TC_BM);
  const int ktiles = kp / TC_BK;
  if (packed) {
    RedqParams P = make_redq(p, 16, 2);
    uint32_t koff = (uint32_t)k;
    FP_CUDA(cudaFuncSetAttribute(k_mm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_mm_tc", st,
              k_mm_tc<1><<<grid, TC_THREADS, smem, st>>>(ma, mb, C, ldc, RW, m, n, nw, ktiles, P, koff,
                                                             ctx->d_err));
    FP_CUDA(cudaGetLastError());
    const int gblocks = ((nw + 7) / 8 + 255) / 256;
    const int gr = (int)std::min<int64_t>((int64_t)m * gblocks, (int64_t)ctx->num_sms * 8);
    FP_LAUNCH(ctx, "k_tc_redq", st, k_tc_redq<<<gr, 256, 0, st>>>(RW, C, ldc, m, n, nw, P, koff % p));
  } else {
    RedqParams P = make_redq(p, 16, 1);
    FP_CUDA(cudaFuncSetAttribute(k_mm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_mm_tc", st,
              k_mm_tc<0><<<grid, TC_THREADS, smem, st>>>(ma, mb, C, ldc, nullptr, m, n, nw, ktiles, P, 0, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
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
