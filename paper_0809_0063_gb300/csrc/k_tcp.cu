// 16-bit matrix products mod p on the tcgen05 tensor cores, persistent and grouped, in two
// forms that share one kernel template:
//
//  packed (RIGHT_TC, right compression, Sec. 7.4), p <= 3: B's columns are paired into one fp16
//    operand word b0 + 2^10 b1 of centred residues (c(0) = 0, c(1) = 1, c(2) = -1), A is
//    converted to centred fp16, so one MMA column accumulates D0 + 2^10 D1 with D0 = sum_l
//    c(a_l) c(b0_l) and D1 likewise: two residues of C per column.  Over a chunk of 448 inner
//    steps both digits stay in (-512, 512) (Eq. lower per chunk, centred), so the fp32 sum is
//    exact and its digits separate.  Each chunk's TMEM accumulator is drained by the epilogue
//    warps into a 32-bit word R = D0 + 2^16 D1 (wrapping, exact since every |digit| <= k <
//    2^15) while the MMA warp fills the other TMEM buffer (delayed reduction, Sec. 2.2).  At the
//    end of a tile an offset k makes both digits of R non-negative and REDQ_2 (Algorithm 2,
//    q = 2^16) recovers them mod p; the residues go straight to C.
//  packed, p = 5, 7: the same with centred residues |c| <= (p-1)/2 and Q = 1023 (p = 5) or 681
//    (p = 7), the largest Q whose pair words are exact fp16 integers; chunks of 64 / 32 inner
//    steps keep both digits below Q / 2, a chunk word's digits are separated by one rounded
//    scaling by 1/Q, and R's 16-bit digits are re-reduced by REDQ every 127 / 113 chunks.  The
//    drains (one per chunk, 128 x 256 values) bound this form, not the MMAs.
//  plain (PLAIN_TC): A and B converted to bf16 (residues < 256 are exact), one residue per
//    column, fp32 sums exact while k (p-1)^2 < 2^24, mod p in the epilogue.  It is the plain
//    product on the same pipe as the packed one.
//
// B is stored MN-major for the MMA (k rows of words or residues), so its conversion is a
// row-by-row map with no transpose; A is K-major.  Schedule: one CTA per SM walks the global
// list of output tiles (128 rows x 256 MMA columns) of up to FP_GROUP_MAX problems, longest
// inner dimension first, with stride gridDim.x.  Roles: warp 0 TMA producer (A 128 x 64 and
// B 64 x 256 per stage, 4-stage ring), warp 1 TMEM allocation (2 x 256 columns) and the
// MMA-issuing thread, warps 2..9 (two per TMEM lane quarter, 128 columns each; for p = 5, 7
// warps 2..17, four per lane quarter, 64 columns each) the accumulator drains, REDQ / mod p and
// the stores, the drains of one tile overlapping the MMAs of the next.  Every wait is bounded (ERR_TIMEOUT on
// give-up, with the drain-and-free exit of the other tensor-core kernels).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fpdqt_internal.cuh"
#include "tc_ptx.cuh"

namespace fpd {

static constexpr int P_BM = 128, P_BNW = 256, P_BK = 64, P_STAGES = 4, P_CHUNK_KT = 7;
static constexpr int P_A_BYTES = P_BM * P_BK * 2;             // 16 KB
static constexpr int P_B_BOX = 64 * P_BK * 2;                 // 8 KB: 64 words x 64 rows
static constexpr int P_B_BYTES = 4 * P_B_BOX;                 // 32 KB
static constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;   // 48 KB
// Epilogue warps: 8 (2 per TMEM lane quarter) for the plain and p <= 3 forms, 16 (4 per lane
// quarter) for p = 5, 7, whose per-chunk drains bound it: twice the warps to hide the TMEM-load
// and arithmetic latency, half the columns (and delayed-reduction words) per thread.  (16 for
// p <= 3 measured slower: 0.456 against 0.50 of bf16, at the 96 registers 18 warps allow.)
__host__ __device__ constexpr int p_epi_warps(int pk) { return pk == 2 ? 16 : 8; }
__host__ __device__ constexpr int p_cw(int pk) { return 4 * P_BNW / p_epi_warps(pk); }   // MMA columns per epilogue thread
__host__ __device__ constexpr int p_threads(int pk) { return 32 * (2 + p_epi_warps(pk)); }
// per epilogue warp: 32 rows x 32 output bytes (row stride 36 bytes: conflict-free word writes)
__host__ __device__ constexpr size_t p_smem(int pk) {
  return 1024 + (size_t)P_STAGES * P_STAGE_BYTES + 256 + (size_t)p_epi_warps(pk) * 32 * 36;
}

// kind::f16, A (K-major) and B (MN-major) both fp16 (ab_type 0) or both bf16 (1), fp32 accumulate.
__host__ __device__ constexpr uint32_t idesc_16_bmn(uint32_t ab_type, int M, int N) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct PProb {
  CUtensorMap ta;    // A16: m rows x kp 16-bit, K-major
  CUtensorMap tb;    // B16: k rows x nw 16-bit (pair words or residues), MN-major
  uint8_t* C;
  int ldc, m, n, nw;
  int ktiles;        // kp / 64
  int nchunks;       // packed: ceil(ktiles / 7); plain: 1
  int tn;            // MMA-column blocks ceil(nw / 256)
  int tile0;
  uint32_t koffset;  // k: added to both digits before REDQ
  uint32_t off_mod_p;
  uint16_t cmma;    // packed p = 5, 7: MMA instructions (16 inner steps each) per chunk
  uint16_t rr;      // packed p = 5, 7: chunks between two re-reductions of R
  uint32_t dmax;    // packed p = 5, 7: largest |digit| one chunk adds
  float qinv;       // packed p = 5, 7: 1 / Q for the pair words c0 + Q c1 (Q = rint(1 / qinv))
  RedqParams P;      // REDQ_2 at q = 2^16
};

// CAP problems per launch: FP_GROUP_MAX for the public calls, P_BATCH_CAP for the large p > 17
// products of an uneven batch.
static constexpr int P_BATCH_CAP = 64;
template <int CAP>
struct PParamsT {
  PProb prob[CAP];
  int nprob;
  int total;
};
using PParams = PParamsT<FP_GROUP_MAX>;
static_assert(sizeof(PParamsT<P_BATCH_CAP>) < 32000, "kernel parameter block limit");

struct PTile {
  const PProb* pr;
  int m0, w0;        // first row, first MMA column
};

template <int CAP>
__device__ __forceinline__ PTile p_tile(const PParamsT<CAP>& g, int t) {
  int i = 0, hi = g.nprob - 1;      // the last problem whose first tile is <= t
  while (i < hi) {
    const int mid = (i + hi + 1) >> 1;
    if (g.prob[mid].tile0 <= t) i = mid;
    else hi = mid - 1;
  }
  const PProb& pr = g.prob[i];
  const int local = t - pr.tile0;
  const int mb = local / pr.tn;
  PTile x;
  x.pr = &pr;
  x.m0 = mb * P_BM;
  x.w0 = (local - mb * pr.tn) * P_BNW;
  return x;
}

// REDQ_2 (Algorithm 2) at q = 2^16 for a compile-time p <= 3, on the words of one thread:
// one division s = floor(w / p), the compression residues u_i = (floor(w / q^i) -
// p floor(s / q^i)) mod q, then one shuffle of a lane-held table indexed by u_0 + p u_1 (the
// Q_2 table of the correction, Sec. 3.4) that returns both final residues at once: byte 0 =
// (u_0 - q u_1 - k) mod p, byte 1 = (u_1 - k) mod p, the offset k (om = k mod p) that made the
// digits non-negative removed in the same lookup.
template <uint32_t PP>
__device__ __forceinline__ uint32_t redq2_pair(uint32_t w, uint32_t table) {
  const uint32_t s = w / PP;
  const uint32_t u0 = (w - PP * s) & 0xFFFFu;
  const uint32_t u1 = ((w >> 16) - PP * (s >> 16)) & 0xFFFFu;
  return __shfl_sync(0xffffffffu, table, u0 + PP * u1) & 0xFFFFu;
}

// This lane's entry of that table: lane = u0 + p u1 < p^2.
__device__ __forceinline__ uint32_t redq2_pair_table(uint32_t p, uint32_t om) {
  const uint32_t lane = threadIdx.x & 31u;
  if (lane >= p * p) return 0;
  const uint32_t u0 = lane % p, u1 = lane / p;
  const uint32_t c = (p - (65536u % p)) % p;           // (-q) mod p
  const uint32_t mu0 = (u0 + c * u1) % p;
  return ((mu0 + p - om) % p) | (((u1 + p - om) % p) << 8);
}

// The end of a packed tile for one thread: its NW words R (= D0 + 2^16 D1 + conversion
// constants, cancelled by `fix`, which also offsets both digits by k >= |digit|) reduced by
// REDQ_2, 2 NW residues stored from dst.  Processed in passes of BW words, each reducing
// R[0..BW-1] and moving R down by BW.  With the divisor, the table and the loop bounds all
// fixed at compile time one unrolled pass over all NW words measured fastest (a rolled
// version with run-time parameters was 1.8x slower: parameters reloaded after every store and
// branches on the correction mode in the inner loop).
static constexpr int P_REDQ_BW = 128;
template <uint32_t PP, int NW, int BW = (NW < P_REDQ_BW ? NW : P_REDQ_BW)>
__device__ __forceinline__ void final_redq(uint32_t (&R)[NW], uint32_t fix, uint32_t table, uint8_t* dst, int c0,
                                           int n, bool in, bool vec) {
  static_assert(BW >= 16 && BW % 16 == 0 && NW % BW == 0, "passes of whole 16-word groups covering R");
#pragma unroll 1
  for (int blk = 0; blk < NW / BW; ++blk) {
#pragma unroll
    for (int h = 0; h < BW / 16; ++h) {        // 16 words -> 32 residues -> two 16-byte stores
      uint32_t o[8];
#pragma unroll
      for (int j = 0; j < 16; j += 2)
        o[j >> 1] = redq2_pair<PP>(R[h * 16 + j] + fix, table) | (redq2_pair<PP>(R[h * 16 + j + 1] + fix, table) << 16);
      uint8_t* d = dst + 2 * (blk * BW + h * 16);
      const int c = c0 + 2 * (blk * BW + h * 16);
      if (vec) {
        reinterpret_cast<uint4*>(d)[0] = make_uint4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<uint4*>(d)[1] = make_uint4(o[4], o[5], o[6], o[7]);
      } else if (in) {
#pragma unroll
        for (int j = 0; j < 32; ++j)   // unrolled: a runtime index into o[] would put it in memory
          if (c + j < n) d[j] = (uint8_t)(o[j >> 2] >> (8 * (j & 3)));
      }
    }
#pragma unroll
    for (int j = 0; j < NW - BW; ++j) R[j] = R[j + BW];
  }
}

// REDQ_2 (Algorithm 2) at q = 2^16 for p = 5, 7 with the correction done by arithmetic (p^2 > 32
// rules out the lane table for p = 7): s = floor(w / p), u_0 = w - p s, u_1 = (floor(w / q) -
// p floor(s / q)) mod q, mu_1 = u_1, mu_0 = (u_0 - q u_1) mod p = (u_0 + c u_1) mod p with
// c = (-q) mod p, both shifted back by the offset (om = offset mod p).  Run-time p (one code
// copy for both primes: these loops run once per tile or per few hundred chunks, and smaller
// code keeps the drain loop and the MMA and TMA loops in the instruction cache).
// Returns mu_0 | mu_1 << 8.
__device__ __forceinline__ uint32_t redq2_arith(uint32_t w, uint32_t om, uint32_t p, uint32_t c, const DivP& dv) {
  const uint32_t s = divp32(w, dv);
  const uint32_t u0 = (w - p * s) & 0xFFFFu;
  const uint32_t u1 = ((w >> 16) - p * (s >> 16)) & 0xFFFFu;
  uint32_t mu1 = u1 + p - om;
  mu1 = mu1 >= p ? mu1 - p : mu1;
  const uint32_t mu0 = modp32(u0 + c * u1 + p - om, dv, p);
  return mu0 | (mu1 << 8);
}

// Every word of R (digits offset to non-negative by `fix`) replaced by its two residues, as a
// word with digits < p: the delayed reduction of Sec. 2.2 applied before a 16-bit digit could
// overflow.  Sixteen words per pass, R rotated by sixteen after each (back in order at the end).
template <int NW>
__device__ __forceinline__ void rereduce_pairs(uint32_t (&R)[NW], uint32_t fix, uint32_t om, uint32_t p, uint32_t c,
                                               const DivP& dv) {
#pragma unroll 1
  for (int pass = 0; pass < NW / 16; ++pass) {
    uint32_t t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t v = redq2_arith(R[j] + fix, om, p, c, dv);
      t[j] = (v & 0xFFu) | ((v >> 8) << 16);
    }
#pragma unroll
    for (int j = 0; j < NW - 16; ++j) R[j] = R[j + 16];
#pragma unroll
    for (int j = 0; j < 16; ++j) R[NW - 16 + j] = t[j];
  }
}

// The end of a packed p = 5, 7 tile: as final_redq, sixteen words (two 16-byte stores) per pass
// with R moved down by sixteen after each.
template <int NW>
__device__ __forceinline__ void final_redq_arith(uint32_t (&R)[NW], uint32_t fix, uint32_t om, uint32_t p, uint32_t c,
                                                 const DivP& dv, uint8_t* dst, int c0, int n, bool in, bool vec) {
#pragma unroll 1
  for (int h = 0; h < NW / 16; ++h) {
    uint32_t o[8];
#pragma unroll
    for (int j = 0; j < 16; j += 2)
      o[j >> 1] = redq2_arith(R[j] + fix, om, p, c, dv) | (redq2_arith(R[j + 1] + fix, om, p, c, dv) << 16);
    uint8_t* d = dst + 32 * h;
    const int cc = c0 + 32 * h;
    if (vec) {
      reinterpret_cast<uint4*>(d)[0] = make_uint4(o[0], o[1], o[2], o[3]);
      reinterpret_cast<uint4*>(d)[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else if (in) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (cc + j < n) d[j] = (uint8_t)(o[j >> 2] >> (8 * (j & 3)));
    }
#pragma unroll
    for (int j = 0; j < NW - 16; ++j) R[j] = R[j + 16];
  }
}

template <int PK, int CAP = FP_GROUP_MAX>
__global__ void __launch_bounds__(p_threads(PK), 1) k_mm_t16(const __grid_constant__ PParamsT<CAP> g, uint32_t* err) {
  constexpr bool PACKED = PK != 0;   // 1: p <= 3 at Q = 2^10; 2: p = 5, 7 at Q = 1023 / 681
  constexpr int P_EPI_WARPS = p_epi_warps(PK), P_CW = p_cw(PK);
  extern __shared__ __align__(1024) uint8_t p_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)p_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + P_STAGES * P_STAGE_BYTES);
  uint64_t* empty = full + P_STAGES;
  uint64_t* tfull = empty + P_STAGES;    // [2] chunk accumulator ready
  uint64_t* tempty = tfull + 2;          // [2] chunk accumulator drained
  uint64_t* drainb = tempty + 2;
  uint64_t* doneb = drainb + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(doneb + 1);
  volatile uint32_t* abort_flag = tmem_slot + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t TMEM_COLS = 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], P_EPI_WARPS);
    }
    mbar_init(drainb, 1);
    mbar_init(doneb, P_EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
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
      uint32_t it = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < g.total && !stop; t += gridDim.x) {
        const PTile x = p_tile(g, t);
        for (int kt = 0; kt < x.pr->ktiles; ++kt, ++it) {
          const int s = (int)(it % P_STAGES);
          if (*abort_flag || !mbar_wait(&empty[s], ((it / P_STAGES) & 1u) ^ 1u, abort_flag)) {
            stop = true;
            break;
          }
          uint8_t* sa = smem + s * P_STAGE_BYTES;
          uint8_t* sb = sa + P_A_BYTES;
          mbar_expect_tx(&full[s], P_STAGE_BYTES);
          tma_load_2d(sa, &x.pr->ta, kt * P_BK, x.m0, &full[s]);
#pragma unroll
          for (int j = 0; j < 4; ++j) tma_load_2d(sb + j * P_B_BOX, &x.pr->tb, x.w0 + 64 * j, kt * P_BK, &full[s]);
        }
      }
      for (uint32_t j = (it > (uint32_t)P_STAGES ? it - P_STAGES : 0u); j < it; ++j)
        mbar_drain(&full[j % P_STAGES], (j / P_STAGES) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0 && PK == 2) {
      // p = 5, 7: a chunk is cmma MMA instructions (16 inner steps each), so chunk boundaries
      // fall inside a k-tile; the stage is released after the k-tile's four instructions
      constexpr uint32_t idesc = idesc_16_bmn(0u, P_BM, P_BNW);
      uint32_t it = 0, gc = 0;      // k tiles and chunks of this CTA so far
      bool stop = false;
      for (int t = blockIdx.x; t < g.total && !stop; t += gridDim.x) {
        const PTile x = p_tile(g, t);
        const int cmma = x.pr->cmma;
        int inchunk = 0;
        uint32_t dtm = tmem;
        for (int kt = 0; kt < x.pr->ktiles && !stop; ++kt, ++it) {
          const int s = (int)(it % P_STAGES);
          if (!mbar_wait(&full[s], (it / P_STAGES) & 1u, abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint8_t* sa = smem + s * P_STAGE_BYTES;
          const uint8_t* sb = sa + P_A_BYTES;
          const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_mn_sw128(sb, P_B_BOX);
          for (int kk = 0; kk < 4; ++kk) {
            if (inchunk == 0) {
              const int buf = (int)(gc & 1u);
              if (gc >= 2 && !mbar_wait(&tempty[buf], ((gc - 2) >> 1) & 1u, abort_flag)) {
                stop = true;
                break;
              }
              tc_fence_after();
              dtm = tmem + (uint32_t)(buf * 256);
            }
            mma_f16(dtm, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 128), idesc, inchunk == 0 ? 0u : 1u);
            if (++inchunk == cmma) {
              mma_commit(&tfull[gc & 1u]);
              inchunk = 0;
              ++gc;
            }
          }
          if (stop) break;
          mma_commit(&empty[s]);
        }
      }
      if (*abort_flag) {
        mma_commit(drainb);
        mbar_drain(drainb, 0);
      }
    } else if (lane == 0) {
      constexpr uint32_t idesc = idesc_16_bmn(PACKED ? 0u : 1u, P_BM, P_BNW);
      uint32_t it = 0, gc = 0;      // k tiles and chunks of this CTA so far
      bool stop = false;
      for (int t = blockIdx.x; t < g.total && !stop; t += gridDim.x) {
        const PTile x = p_tile(g, t);
        int kt = 0;
        for (int c = 0; c < x.pr->nchunks && !stop; ++c, ++gc) {
          const int buf = (int)(gc & 1u);
          if (gc >= 2 && !mbar_wait(&tempty[buf], ((gc - 2) >> 1) & 1u, abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t dtm = tmem + (uint32_t)(buf * 256);
          const int kend = PACKED ? min(x.pr->ktiles, kt + P_CHUNK_KT) : x.pr->ktiles;
          bool first = true;
          for (; kt < kend; ++kt, ++it) {
            const int s = (int)(it % P_STAGES);
            if (!mbar_wait(&full[s], (it / P_STAGES) & 1u, abort_flag)) {
              stop = true;
              break;
            }
            tc_fence_after();
            const uint8_t* sa = smem + s * P_STAGE_BYTES;
            const uint8_t* sb = sa + P_A_BYTES;
            const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_mn_sw128(sb, P_B_BOX);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // K = 16: A +32 bytes in the row, B +16 rows of 128 bytes
              mma_f16(dtm, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 128), idesc, first ? 0u : 1u);
              first = false;
            }
            mma_commit(&empty[s]);
          }
          if (!stop) mma_commit(&tfull[buf]);
        }
      }
      if (*abort_flag) {
        mma_commit(drainb);
        mbar_drain(drainb, 0);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ drains, REDQ / mod p, stores (warps 2..)
    const int q = warp & 3;                      // TMEM lane quarter
    const int part = (warp - 2) >> 2;            // MMA columns part * P_CW .. + P_CW - 1
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint32_t* const epi_stage =                 // this warp's 32 x 36-byte store buffer
        reinterpret_cast<uint32_t*>(smem + P_STAGES * P_STAGE_BYTES + 256) + (warp - 2) * (32 * 9);
    uint32_t gc = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < g.total && ok && !PACKED; t += gridDim.x, ++gc) {
      // plain: one accumulator per tile, mod p of each fp32 sum (an exact integer)
      const PTile x = p_tile(g, t);
      const PProb& pr = *x.pr;
      const int buf = (int)(gc & 1u);
      uint32_t got = 1;
      if (lane == 0) got = mbar_wait(&tfull[buf], (gc >> 1) & 1u, abort_flag) ? 1u : 0u;
      if (!__shfl_sync(0xffffffffu, got, 0)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const DivP dv = pr.P.dv;
      const uint32_t p = pr.P.p;
      const int row = x.m0 + q * 32 + lane;
      for (int cb = 0; cb < P_CW / 32; ++cb) {
        const int col0 = part * P_CW + cb * 32;
        uint32_t v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * 256 + col0), v);
        uint32_t o[8];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          uint32_t w = 0;
#pragma unroll
          for (int u = 0; u < 4; ++u) w |= modp32(__float2uint_rn(__uint_as_float(v[j + u])), dv, p) << (8 * u);
          o[j >> 2] = w;
        }
        const int c0 = x.w0 + col0;                 // the same for the whole warp
        uint8_t* dst = pr.C + (size_t)row * pr.ldc + c0;
        const bool vec = row < pr.m && c0 + 32 <= pr.n && ((((uintptr_t)dst) & 15u) == 0);
        if (__all_sync(0xffffffffu, vec)) {
          reinterpret_cast<uint4*>(dst)[0] = make_uint4(o[0], o[1], o[2], o[3]);
          reinterpret_cast<uint4*>(dst)[1] = make_uint4(o[4], o[5], o[6], o[7]);
        } else if (c0 < pr.n) {
          // rows not 16-byte aligned or a ragged edge: the warp's 32 rows x 32 bytes go through
          // shared memory and out one row at a time, the 32 lanes on consecutive bytes
#pragma unroll
          for (int j = 0; j < 8; ++j) epi_stage[lane * 9 + j] = o[j];
          __syncwarp();
          const uint8_t* sb = reinterpret_cast<const uint8_t*>(epi_stage);
          const int r0 = x.m0 + q * 32;
          const bool col_in = c0 + lane < pr.n;
          for (int r = 0; r < 32 && r0 + r < pr.m; ++r)
            if (col_in) pr.C[(size_t)(r0 + r) * pr.ldc + c0 + lane] = sb[r * 36 + lane];
          __syncwarp();
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
    for (int t = blockIdx.x; t < g.total && ok && PK == 2; t += gridDim.x) {
      // p = 5, 7: chunk words v = d0 + Q d1 with |d0|, |d1| <= dmax < Q / 2; every
      // chunk is moved into R = D0 + 2^16 D1 as below, and every rr chunks R's digits are
      // replaced by their residues before a 16-bit digit could overflow
      const PTile x = p_tile(g, t);
      const PProb& pr = *x.pr;
      uint32_t R[P_CW];
#pragma unroll
      for (int j = 0; j < P_CW; ++j) R[j] = 0;
      const uint32_t p = pr.P.p, dmax = pr.dmax, rr = (uint32_t)pr.rr;
      const float qinv = pr.qinv;
      const uint32_t qdec = 65536u - (uint32_t)rintf(1.0f / qinv);
      const uint32_t cmag = 0x4B400000u * (1u + qdec);   // added to every R word per chunk
      uint32_t cr = 0;     // chunks added since R last held residues
      for (int c = 0; c < pr.nchunks; ++c, ++gc) {
        const int buf = (int)(gc & 1u);
        uint32_t got = 1;
        if (lane == 0) got = mbar_wait(&tfull[buf], (gc >> 1) & 1u, abort_flag) ? 1u : 0u;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
        tc_fence_after();
        // 1.5 2^23 added: the float's bits are y = 0x4B400000 + v exactly; the same after
        // scaling by 1/Q gives t = 0x4B400000 + round(v / Q) = 0x4B400000 + d1 (|d0| / Q <= 0.43,
        // far from the rounding boundary), and y + (2^16 - Q) t = d0 + 2^16 d1 + cmag with the
        // per-chunk constant cmag = 0x4B400000 (1 + 2^16 - Q) (mod 2^32), removed by `fix`
        const uint32_t base = tmem + lane_base + (uint32_t)(buf * 256 + part * P_CW);
        uint32_t va[16], vb[16];
        tmem_ld16_nowait(base, va);
        tmem_wait();
#pragma unroll
        for (int blk = 0; blk < P_CW / 16; ++blk) {
          if (blk + 1 < P_CW / 16) {
            if (blk & 1) tmem_ld16_nowait(base + (uint32_t)((blk + 1) * 16), va);
            else tmem_ld16_nowait(base + (uint32_t)((blk + 1) * 16), vb);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float v = __uint_as_float((blk & 1) ? vb[j] : va[j]);
            const uint32_t y = (uint32_t)__float_as_int(v + 12582912.0f);
            const uint32_t t1 = (uint32_t)__float_as_int(fmaf(v, qinv, 12582912.0f));
            R[blk * 16 + j] += y + t1 * qdec;
          }
          tmem_wait();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        if (++cr == rr && c + 1 < pr.nchunks) {
          const uint32_t off = dmax * cr;
          const uint32_t fix = off * 65537u - cr * cmag;
          rereduce_pairs<P_CW>(R, fix, off % p, p, pr.P.c, pr.P.dv);
          cr = 0;
        }
      }
      if (!ok) break;
      const uint32_t off = dmax * cr;
      const uint32_t fix = off * 65537u - cr * cmag;
      const int row = x.m0 + q * 32 + lane;
      const int c0 = 2 * (x.w0 + part * P_CW);
      const int n = pr.n;
      const bool in = row < pr.m && c0 < n;
      uint8_t* dst = pr.C + (size_t)row * pr.ldc + c0;
      const bool vec = in && c0 + 2 * P_CW <= n && ((((uintptr_t)dst) & 15u) == 0);
      final_redq_arith<P_CW>(R, fix, off % p, p, pr.P.c, pr.P.dv, dst, c0, n, in, vec);
    }
    for (int t = blockIdx.x; t < g.total && ok && PK == 1; t += gridDim.x) {
      const PTile x = p_tile(g, t);
      const PProb& pr = *x.pr;
      uint32_t R[P_CW];   // unsigned: wraps modulo 2^32 (the conversion offsets cancel at the end)
#pragma unroll
      for (int j = 0; j < P_CW; ++j) R[j] = 0;
      for (int c = 0; c < pr.nchunks; ++c, ++gc) {
        const int buf = (int)(gc & 1u);
        // one lane waits, the warp follows: the tcgen05.ld below and the shuffles of REDQ need
        // all 32 lanes on the same path even if the wait gives up
        uint32_t got = 1;
        if (lane == 0) got = mbar_wait(&tfull[buf], (gc >> 1) & 1u, abort_flag) ? 1u : 0u;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
        tc_fence_after();
        // blocks of 16 columns, loads double-buffered.  Chunk word v = d0 + 2^10 d1 with
        // |d0|, |d1| < 512: adding 1.5 2^23 makes the float's bits 0x4B400000 + v exactly, so
        // y - 0x4B400000 = v with no conversion instruction; d1 = round(v / 2^10).
        const uint32_t base = tmem + lane_base + (uint32_t)(buf * 256 + part * P_CW);
        uint32_t va[16], vb[16];
        tmem_ld16_nowait(base, va);
        tmem_wait();
#pragma unroll
        for (int blk = 0; blk < P_CW / 16; ++blk) {
          if (blk + 1 < P_CW / 16) {
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
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      if (!ok) break;
      // R = D0 + 2^16 D1 (+ the per-chunk constants); offset both digits by k, REDQ_2, store
      // parameters copied to registers (read through the grid-constant block they would be
      // reloaded after every store to C)
      const uint32_t fix = pr.koffset * 65537u - (uint32_t)pr.nchunks * 0x4B400000u;
      const uint32_t p = pr.P.p;
      const uint32_t table = redq2_pair_table(p, pr.off_mod_p);
      const int row = x.m0 + q * 32 + lane;
      const int c0 = 2 * (x.w0 + part * P_CW);   // first column of C for this thread
      const int n = pr.n;
      const bool in = row < pr.m && c0 < n;
      uint8_t* dst = pr.C + (size_t)row * pr.ldc + c0;
      const bool vec = in && c0 + 2 * P_CW <= n && ((((uintptr_t)dst) & 15u) == 0);
      if (p == 3) final_redq<3, P_CW>(R, fix, table, dst, c0, n, in, vec);
      else final_redq<2, P_CW>(R, fix, table, dst, c0, n, in, vec);
    }
    __syncwarp();
    tc_fence_before();
    if (lane == 0) mbar_arrive(doneb);
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) flag_error(err, ERR_TIMEOUT);
  if (warp == 1) {
    if (lane == 0) mbar_drain(doneb, 0);
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// bf16 bits of a residue v <= 255: the float 2^23 + v has v in its low mantissa bits, so
// subtracting 2^23 gives float(v) exactly; its top 16 bits are the bf16 (exact, 8 bits).
__device__ __forceinline__ uint32_t bf16_of(uint32_t v) {
  return __float_as_uint(__uint_as_float(0x4B000000u | v) - 8388608.0f) >> 16;
}

// A16[r][c] (m x kp, zero padded) = centred fp16 (PACKED) or bf16 of A[r][c]; one thread per
// 16 columns.  Residues >= p set ERR_RANGE.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_t16_convert_a(const uint8_t* __restrict__ A, int lda, uint16_t* __restrict__ dst,
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
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
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
      uint32_t o[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bad |= __vcmpgeu4(w[q], 0x01010101u * p);
        const uint32_t x = w[q];
        if (PACKED && p <= 3) {
          o[2 * q] = h16_centred(x & 0xffu) | (h16_centred((x >> 8) & 0xffu) << 16);
          o[2 * q + 1] = h16_centred((x >> 16) & 0xffu) | (h16_centred(x >> 24) << 16);
        } else if (PACKED) {   // p = 5, 7: centred residues in [-(p-1)/2, (p-1)/2]
          o[2 * q] = h16_centred_p(x & 0xffu, p) | (h16_centred_p((x >> 8) & 0xffu, p) << 16);
          o[2 * q + 1] = h16_centred_p((x >> 16) & 0xffu, p) | (h16_centred_p(x >> 24, p) << 16);
        } else {
          o[2 * q] = bf16_of(x & 0xffu) | (bf16_of((x >> 8) & 0xffu) << 16);
          o[2 * q + 1] = bf16_of((x >> 16) & 0xffu) | (bf16_of(x >> 24) << 16);
        }
      }
      uint4* d = reinterpret_cast<uint4*>(dst + (size_t)r * kp + c0);
      d[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// B16 (k x ldw 16-bit, zero past nw) row by row from B (k x n), no transpose.  PACKED: word
// j = fp16 of c(B[l][2j]) + Q c(B[l][2j+1]) (Q = 2^10 for p <= 3, 1023 / 681 for p = 5 / 7; the second
// residue 0 past column n), one
// thread per 16 bytes of B (8 words); plain: bf16 of B[l][j], one thread per 8 bytes of B
// (8 elements).  Residues >= p set ERR_RANGE.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_t16_convert_b(const uint8_t* __restrict__ B, int ldb, uint16_t* __restrict__ dst,
                                                       int k, int n, int ldw, uint32_t p, uint32_t* err) {
  constexpr int IN = PACKED ? 16 : 8;            // input bytes per thread (8 output words)
  const int groups = ldw >> 3;
  uint32_t bad = 0;
  const bool vec = (((uintptr_t)B) & (IN - 1)) == 0 && (ldb & (IN - 1)) == 0;
  const uint32_t pp = 0x01010101u * p;
  for (int r = blockIdx.x; r < k; r += gridDim.x)
    for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
      const int c0 = gi * IN;                    // first byte column of B
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      const uint8_t* src = B + (size_t)r * ldb + c0;
      if (vec && c0 + IN <= n) {
        if (PACKED) {
          const uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
          w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
        } else {
          const uint2 x = __ldg(reinterpret_cast<const uint2*>(src));
          w[0] = x.x; w[1] = x.y;
        }
      } else if (c0 < n) {
#pragma unroll
        for (int q = 0; q < IN / 4; ++q) {
          uint32_t t = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) t |= (uint32_t)(c0 + 4 * q + j < n ? src[4 * q + j] : 0) << (8 * j);
          w[q] = t;
        }
      }
      uint32_t o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bad |= __vcmpgeu4(w[q], pp);
        const uint32_t x = w[q];
        if (PACKED && p <= 3) {
          o[q] = h16_pair_word(x & 0xffu, (x >> 8) & 0xffu) | (h16_pair_word((x >> 16) & 0xffu, x >> 24) << 16);
        } else if (PACKED) {   // p = 5, 7: c(b0) + Q c(b1), Q = 1023 / 681
          const float Q = p == 5 ? 1023.0f : 681.0f;
          o[q] = h16_pair_word_p(x & 0xffu, (x >> 8) & 0xffu, p, Q) |
                 (h16_pair_word_p((x >> 16) & 0xffu, x >> 24, p, Q) << 16);
        } else {
          const uint32_t y = w[q >> 1] >> (16 * (q & 1));
          o[q] = bf16_of(y & 0xffu) | (bf16_of((y >> 8) & 0xffu) << 16);
        }
      }
      *reinterpret_cast<uint4*>(dst + (size_t)r * ldw + gi * 8) = make_uint4(o[0], o[1], o[2], o[3]);
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// ---------------------------------------------------------------- host side

// Packed fp16 words: p <= 3 at Q = 2^10 in chunks of 448 inner steps (k <= 32767 keeps R's
// 16-bit digits from overflowing without re-reduction); p = 5, 7 at the largest Q whose pair
// words stay exact in fp16 with centred residues |c| <= (p-1)/2 ((p-1)/2 (1 + Q) <= 2048: Q =
// 1023 for p = 5, 681 for p = 7), in chunks of 64 (p = 5) or 32 (p = 7) inner steps so that
// every chunk digit stays below Q / 2 in magnitude (256 < 511.5, 288 < 340.5).
bool f16p_ok(uint32_t p, int k) { return (p <= 3 && k <= 32767) || p == 5 || p == 7; }

// Chunk parameters of the p = 5, 7 packed form: Q, MMA instructions per chunk, the largest
// |digit| a chunk adds ((p-1)/2)^2 per inner step, and the chunks R takes before its 16-bit
// digits could overflow ((p-1) + 2 dmax rr < 2^16).
static void pk2_params(uint32_t p, uint32_t* Q, int* cmma, uint32_t* dmax, int* rr) {
  const uint32_t h = (p - 1) / 2;
  *Q = p == 5 ? 1023u : 681u;
  *cmma = p == 5 ? 4 : 2;
  *dmax = h * h * 16u * (uint32_t)*cmma;
  *rr = (int)((65535u - (p - 1)) / (2u * *dmax));
}

// Convert the problems' operands into context scratch and launch the grouped kernel(s); the
// caller holds the context lock.  Every problem passed fp_matmul's checks and the variant's
// exactness rule (packed: f16p_ok; plain: k (p-1)^2 < 2^24).
static fp_status launch_t16_mode(fp_ctx ctx, const std::vector<const fp_mm_problem*>& v, int pk, cudaStream_t st);

static fp_status launch_t16_locked(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, bool packed,
                                   cudaStream_t st) {
  // packed problems run in two kernels: p <= 3 (mode 1) and p = 5, 7 (mode 2)
  std::vector<const fp_mm_problem*> v1, v2;
  for (size_t i = 0; i < count; ++i) (packed && pr[i]->p > 3 ? v2 : v1).push_back(pr[i]);
  fp_status s = v1.empty() ? FP_OK : launch_t16_mode(ctx, v1, packed ? 1 : 0, st);
  if (s == FP_OK && !v2.empty()) s = launch_t16_mode(ctx, v2, 2, st);
  return s;
}

static fp_status launch_t16_mode(fp_ctx ctx, const std::vector<const fp_mm_problem*>& v0, int pk, cudaStream_t st) {
  const bool packed = pk != 0;
  std::vector<const fp_mm_problem*> v(v0);
  std::stable_sort(v.begin(), v.end(), [](const fp_mm_problem* a, const fp_mm_problem* b) { return a->k > b->k; });
  auto words = [packed](int n) { return packed ? (n + 1) / 2 : n; };
  for (size_t base = 0; base < v.size(); base += FP_GROUP_MAX) {
    const int cnt = (int)std::min<size_t>(FP_GROUP_MAX, v.size() - base);
    // scratch layout: per problem A16 (m x kp) then B16 (k x ldw), 1024-byte aligned
    size_t off[FP_GROUP_MAX][2], total = 0;
    for (int i = 0; i < cnt; ++i) {
      const fp_mm_problem& x = *v[base + i];
      const size_t kp = (size_t)(x.k + P_BK - 1) / P_BK * P_BK, ldw = ((size_t)words(x.n) + 7) / 8 * 8;
      off[i][0] = total;
      total += (x.m * kp * 2 + 1023) & ~(size_t)1023;
      off[i][1] = total;
      total += (x.k * ldw * 2 + 1023) & ~(size_t)1023;
    }
    fp_status s = ensure_scratch(ctx, total + 1024, 0, st);
    if (s != FP_OK) return s;
    PParams hp;
    std::memset(&hp, 0, sizeof hp);
    int tile = 0;
    for (int i = 0; i < cnt; ++i) {
      const fp_mm_problem& x = *v[base + i];
      const int kp = (x.k + P_BK - 1) / P_BK * P_BK, nw = words(x.n), ldw = (nw + 7) / 8 * 8;
      uint16_t* A16 = (uint16_t*)((uint8_t*)ctx->scratch + off[i][0]);
      uint16_t* B16 = (uint16_t*)((uint8_t*)ctx->scratch + off[i][1]);
      const int ga = std::min(x.m, ctx->num_sms * 16), gb = std::min(x.k, ctx->num_sms * 16);
      if (packed) {
        FP_LAUNCH(ctx, "k_t16_convert_a", st,
                  k_t16_convert_a<true><<<ga, 256, 0, st>>>(x.A, x.lda, A16, x.m, x.k, kp, x.p, ctx->d_err));
        FP_LAUNCH(ctx, "k_t16_convert_b", st,
                  k_t16_convert_b<true><<<gb, 256, 0, st>>>(x.B, x.ldb, B16, x.k, x.n, ldw, x.p, ctx->d_err));
      } else {
        FP_LAUNCH(ctx, "k_t16_convert_a", st,
                  k_t16_convert_a<false><<<ga, 256, 0, st>>>(x.A, x.lda, A16, x.m, x.k, kp, x.p, ctx->d_err));
        FP_LAUNCH(ctx, "k_t16_convert_b", st,
                  k_t16_convert_b<false><<<gb, 256, 0, st>>>(x.B, x.ldb, B16, x.k, x.n, ldw, x.p, ctx->d_err));
      }
      FP_CUDA(cudaGetLastError());
      PProb& g = hp.prob[i];
      s = make_map_ld(&g.ta, A16, (uint64_t)x.m, (uint64_t)kp, (uint64_t)kp, P_BM, 2);
      if (s != FP_OK) return s;
      s = make_map_ld(&g.tb, B16, (uint64_t)x.k, (uint64_t)nw, (uint64_t)ldw, 64, 2);
      if (s != FP_OK) return s;
      g.C = x.C;
      g.ldc = x.ldc;
      g.m = x.m;
      g.n = x.n;
      g.nw = nw;
      g.ktiles = kp / P_BK;
      g.nchunks = packed ? (g.ktiles + P_CHUNK_KT - 1) / P_CHUNK_KT : 1;
      if (pk == 2) {
        uint32_t Q = 0;
        int cmma = 0, rr = 0;
        pk2_params(x.p, &Q, &cmma, &g.dmax, &rr);
        g.cmma = (uint16_t)cmma;
        g.rr = (uint16_t)rr;
        g.nchunks = g.ktiles * 4 / cmma;
        g.qinv = 1.0f / (float)Q;
      }
      g.tn = (nw + P_BNW - 1) / P_BNW;
      g.tile0 = tile;
      g.koffset = (uint32_t)x.k;
      g.off_mod_p = (uint32_t)x.k % x.p;
      g.P = make_redq(x.p, 16, packed ? 2 : 1);
      tile += ((x.m + P_BM - 1) / P_BM) * g.tn;
    }
    hp.nprob = cnt;
    hp.total = tile;
    const int grid = std::min(tile, ctx->num_sms);
    if (pk == 2) {
      FP_CUDA(cudaFuncSetAttribute(k_mm_t16<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem(2)));
      FP_LAUNCH(ctx, "k_mm_t16_packed_p57", st, k_mm_t16<2><<<grid, p_threads(2), p_smem(2), st>>>(hp, ctx->d_err));
    } else if (packed) {
      FP_CUDA(cudaFuncSetAttribute(k_mm_t16<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem(1)));
      FP_LAUNCH(ctx, "k_mm_t16_packed", st, k_mm_t16<1><<<grid, p_threads(1), p_smem(1), st>>>(hp, ctx->d_err));
    } else {
      FP_CUDA(cudaFuncSetAttribute(k_mm_t16<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem(0)));
      FP_LAUNCH(ctx, "k_mm_t16_plain", st, k_mm_t16<0><<<grid, p_threads(0), p_smem(0), st>>>(hp, ctx->d_err));
    }
    FP_CUDA(cudaGetLastError());
  }
  return FP_OK;
}

// ---------------------------------------------------------------- plain products of an uneven batch

// One conversion job: rows of `row_bytes` residue bytes at src (leading dimension src_ld) to bf16
// at dst (leading dimension dst_ld elements, dst 16-byte aligned, dst_ld a multiple of 4).
static constexpr uint32_t JOB_SMEM_MAX = 8192;   // 64 KB of first rows

struct T16Job {
  const uint8_t* src;
  uint16_t* dst;
  uint32_t row_bytes, src_ld, dst_ld, p;
  uint64_t row0;      // first row of this job in the launch's flat row numbering
};

// One warp per row of all jobs: four residues per lane and step (read as the aligned source
// words that hold them, never past the row's last byte's word), range-checked, written as four
// bf16.  Bytes past the row are masked to 0 (their bf16 lands in the row's padding, which the
// tensor maps' extents exclude).
__global__ void __launch_bounds__(256) k_t16_convert_jobs(const T16Job* __restrict__ jobs, uint32_t njobs,
                                                          uint64_t rows, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t bad = 0;
  // the jobs' first rows in shared memory (when they fit the launch's dynamic allocation) so
  // that the per-row search for its job stays on chip
  extern __shared__ uint64_t s_row0[];
  const bool in_smem = njobs <= JOB_SMEM_MAX;
  if (in_smem)
    for (uint32_t i = threadIdx.x; i < njobs; i += blockDim.x) s_row0[i] = jobs[i].row0;
  __syncthreads();
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    uint32_t lo = 0, hi = njobs - 1;             // the last job with row0 <= r
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if ((in_smem ? s_row0[mid] : jobs[mid].row0) <= r) lo = mid;
      else hi = mid - 1;
    }
    const T16Job J = jobs[lo];
    const uint64_t row = r - J.row0;
    const uint8_t* src = J.src + row * J.src_ld;
    uint2* dst = reinterpret_cast<uint2*>(J.dst + row * J.dst_ld);
    const uint32_t off = (uint32_t)((uintptr_t)src & 3u);
    const uint32_t* base = reinterpret_cast<const uint32_t*>(src - off);
    const uint32_t pk = 0x01010101u * (128u - J.p);
    const uint32_t nw = (J.row_bytes + 3) / 4;
    for (uint32_t c = lane; c < nw; c += 32) {
      const uint32_t a0 = base[c];
      const uint32_t a1 = (off != 0 && 4 * c + 4 - off < J.row_bytes) ? base[c + 1] : 0u;
      uint32_t w = off ? __funnelshift_r(a0, a1, 8 * off) : a0;
      const uint32_t nb = J.row_bytes - 4 * c;
      if (nb < 4) w &= (1u << (8 * nb)) - 1u;
      bad |= w | ((w & 0x7F7F7F7Fu) + (pk & 0x7F7F7F7Fu));
      dst[c] = make_uint2(bf16_of(w & 0xffu) | (bf16_of((w >> 8) & 0xffu) << 16),
                          bf16_of((w >> 16) & 0xffu) | (bf16_of(w >> 24) << 16));
    }
  }
  if (bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

// Plain products (k (p-1)^2 < 2^24, p <= 251) of an uneven batch: operands converted to bf16 in
// one launch into `scratch` (at least t16_batch_bytes(...) bytes, 1024-byte aligned), then grouped
// launches of up to P_BATCH_CAP products.  The caller holds the context lock.
static uint64_t t16_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t t16_batch_bytes(const fp_mm_problem* const* pr, size_t count) {
  uint64_t bytes = t16_up(count * 2 * sizeof(T16Job), 1024);
  for (size_t i = 0; i < count; ++i) {
    const fp_mm_problem& x = *pr[i];
    bytes += t16_up((uint64_t)x.m * t16_up(x.k, P_BK) * 2, 1024) + t16_up((uint64_t)x.k * t16_up(x.n, 8) * 2, 1024);
  }
  return bytes;
}

fp_status launch_mm_t16_plain_batch(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, uint8_t* scratch,
                                    cudaStream_t st) {
  std::vector<const fp_mm_problem*> v(pr, pr + count);
  std::stable_sort(v.begin(), v.end(), [](const fp_mm_problem* a, const fp_mm_problem* b) { return a->k > b->k; });
  std::vector<T16Job> jobs;
  std::vector<uint16_t*> a16(v.size()), b16(v.size());
  uint64_t off = t16_up(v.size() * 2 * sizeof(T16Job), 1024), rows = 0;
  for (size_t i = 0; i < v.size(); ++i) {
    const fp_mm_problem& x = *v[i];
    const uint64_t kp = t16_up(x.k, P_BK), ldw = t16_up(x.n, 8);
    a16[i] = (uint16_t*)(scratch + off);
    off += t16_up((uint64_t)x.m * kp * 2, 1024);
    b16[i] = (uint16_t*)(scratch + off);
    off += t16_up((uint64_t)x.k * ldw * 2, 1024);
    jobs.push_back(T16Job{x.A, a16[i], (uint32_t)x.k, (uint32_t)x.lda, (uint32_t)kp, x.p, rows});
    rows += x.m;
    jobs.push_back(T16Job{x.B, b16[i], (uint32_t)x.n, (uint32_t)x.ldb, (uint32_t)ldw, x.p, rows});
    rows += x.k;
  }
  fp_status s = upload_staged(ctx, 2, scratch, jobs.data(), jobs.size() * sizeof(T16Job), st);
  if (s != FP_OK) return s;
  const int cgrid = (int)std::min<uint64_t>((rows + 7) / 8, (uint64_t)ctx->num_sms * 8);
  const size_t jsm = std::min<size_t>(jobs.size(), JOB_SMEM_MAX) * sizeof(uint64_t);
  FP_CUDA(cudaFuncSetAttribute(k_t16_convert_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(JOB_SMEM_MAX * 8)));
  FP_LAUNCH(ctx, "k_t16_convert_jobs", st,
            k_t16_convert_jobs<<<cgrid, 256, jsm, st>>>((const T16Job*)scratch, (uint32_t)jobs.size(), rows, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  FP_CUDA(cudaFuncSetAttribute(k_mm_t16<0, P_BATCH_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem(0)));
  for (size_t base = 0; base < v.size(); base += P_BATCH_CAP) {
    const int cnt = (int)std::min<size_t>(P_BATCH_CAP, v.size() - base);
    PParamsT<P_BATCH_CAP> hp;
    std::memset(&hp, 0, sizeof hp);
    int tile = 0;
    for (int i = 0; i < cnt; ++i) {
      const fp_mm_problem& x = *v[base + i];
      const uint64_t kp = t16_up(x.k, P_BK), ldw = t16_up(x.n, 8);
      PProb& g = hp.prob[i];
      // extents k and n: the pad columns past them are never read (the TMA fills zeros)
      s = make_map_ld(&g.ta, a16[base + i], (uint64_t)x.m, (uint64_t)x.k, kp, P_BM, 2);
      if (s != FP_OK) return s;
      s = make_map_ld(&g.tb, b16[base + i], (uint64_t)x.k, (uint64_t)x.n, ldw, 64, 2);
      if (s != FP_OK) return s;
      g.C = x.C;
      g.ldc = x.ldc;
      g.m = x.m;
      g.n = x.n;
      g.nw = x.n;
      g.ktiles = (int)(kp / P_BK);
      g.nchunks = 1;
      g.tn = (x.n + P_BNW - 1) / P_BNW;
      g.tile0 = tile;
      g.koffset = (uint32_t)x.k;
      g.off_mod_p = (uint32_t)x.k % x.p;
      g.P = make_redq(x.p, 16, 1);
      tile += ((x.m + P_BM - 1) / P_BM) * g.tn;
    }
    hp.nprob = cnt;
    hp.total = tile;
    const int grid = std::min(tile, ctx->num_sms);
    FP_LAUNCH(ctx, "k_mm_t16_plain", st, (k_mm_t16<0, P_BATCH_CAP><<<grid, p_threads(0), p_smem(0), st>>>(hp, ctx->d_err)));
    FP_CUDA(cudaGetLastError());
  }
  return FP_OK;
}

fp_status launch_mm_t16_direct(fp_ctx ctx, const fp_mm_problem& x, bool packed, cudaStream_t st) {
  const fp_mm_problem* one = &x;
  return launch_t16_locked(ctx, &one, 1, packed, st);
}

fp_status launch_mm_t16_grouped(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, bool packed,
                                cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return launch_t16_locked(ctx, pr, count, packed, st);
}

}  // namespace fpd
