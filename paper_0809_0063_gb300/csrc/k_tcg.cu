// Grouped, persistent plain product C = A B mod p on the tcgen05 tensor cores with e4m3
// operands (kind::f8f6f4, fp32 accumulation in TMEM) for several independent problems in one
// launch.
//
// Residues 0..16 read as e4m3 bit patterns are exactly r 2^-9 (codes 0..7 are subnormals
// m 2^-9, codes 8..15 the binade [2^-6, 2^-5) with step 2^-9, code 16 is 2^-5), so the
// caller's uint8 arrays are the MMA operands as they stand: A K-major (rows of k bytes), B
// MN-major (rows of n bytes, one per k).  Each fp32 sum is 2^-18 times the integer sum
// sum_l a_il b_lj, exact while that integer stays below 2^24 (k (p-1)^2 < 2^24); the epilogue
// scales it back by 2^18 and reduces it mod p (delayed reduction, Sec. 2.2, with a single
// reduction at the end).
//
// Persistent schedule: one CTA per SM walks the global list of 128 x 256 output tiles (all
// problems, those with the longest inner dimension first) in waves of gridDim.x tiles, taken in
// forward order in even waves and reversed in odd ones (better balance than a plain stride when
// the tiles' lengths differ: 0.98 vs 0.94 of the mean load for the matrix step).  Roles:
//   warp 0       producer: computes each tile's parameters once (the next tile's while the
//                current tile's copies are issued) and hands them to the other roles through a
//                4-slot ring in shared memory; per k tile, A 128 x 128 bytes and B two boxes of
//                128 x 128 bytes (128-byte swizzle) into the stage ring (4 stages; TMA from the
//                caller's arrays, or 3 stages of plain bulk copies of pre-tiled operands),
//   warp 1       TMEM allocation (512 columns = two 128 x 256 fp32 accumulators) and the
//                single MMA-issuing thread; tile i accumulates into buffer i & 1,
//   warps 2..    epilogue of tile i (tcgen05.ld, scale, mod p, stores: 16-byte stores where a
//                row is 16-byte aligned, else through a small per-warp buffer with the lanes
//                on consecutive bytes of a row) while the MMAs of tile i + 1 run into the other
//                buffer; 2 (TMA problems) or 4 (pre-tiled) warps per TMEM lane quarter, taking
//                its 32-column blocks in turn (pre-tiled: all of a warp's blocks are reduced
//                into shared memory and the accumulator released before the stores).  Before
//                waiting for a tile's accumulator they range-check a slice of its inputs with
//                plain global loads (off the shared-memory pipeline): the A panel of (problem,
//                row block) is used by the tiles of every column block and the B panel of
//                (problem, column block) by those of every row block, so the tile in column
//                block nb checks slice nb of its A panel and the tile in row block mb slice mb of
//                its B panel: every input byte is checked exactly once (pre-tiled operands were
//                checked when packed).
// A stage is released when the MMAs that read it have completed (tcgen05.commit).  Every wait
// is bounded: a wait that gives up sets the abort flag, the roles stop, in-flight copies and MMAs
// are drained, TMEM is freed and the context's sticky flag reports ERR_TIMEOUT.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fpdqt_internal.cuh"
#include "tc_ptx.cuh"

namespace fpd {

static constexpr int G_BM = 128, G_BN = 256, G_BK = 128, G_STAGES = 4;
static constexpr int G_A_BYTES = G_BM * G_BK;                 // 16 KB
static constexpr int G_B_BYTES = G_BN * G_BK;                 // 32 KB (two 128-column boxes)
static constexpr int G_STAGE_BYTES = G_A_BYTES + G_B_BYTES;   // 48 KB
// epilogue warps: 2 per TMEM lane quarter for TMA problems (long tiles, the epilogue hidden
// behind the MMAs), 4 for pre-tiled ones (short tiles of uneven batches: the epilogue is
// latency-bound and more warps hide more of it; 8, 12, 16 warps: 0.58, 0.556, 0.486 ms on the
// benchmark batch, the last with the stores after the accumulator's release)
__host__ __device__ constexpr int g_epi_warps(bool pre) { return pre ? 16 : 8; }
__host__ __device__ constexpr int g_threads(bool pre) { return 64 + 32 * g_epi_warps(pre); }
// Shared memory: the stage ring, barriers, tmem address and abort flag (G_BAR_BYTES), the tile
// parameter ring (G_RING_BYTES), the epilogue warps' store buffers (32 rows x 36 bytes each: row
// stride 9 words, conflict-free), then (pre-tiled launches) the problems' first tiles and
// column-block counts.
static constexpr int G_STAGES_PRE = 3;
static constexpr int G_BAR_BYTES = 256, G_RING_BYTES = 512;
__host__ __device__ constexpr int g_stages(bool pre) { return pre ? G_STAGES_PRE : G_STAGES; }
// 32 x 32-byte blocks each epilogue warp stages at once: pre-tiled, all of a tile's (8 blocks per
// lane quarter shared by g_epi_warps / 4 warps)
__host__ __device__ constexpr int g_stage_blocks(bool pre) {
  return pre ? (8 + g_epi_warps(pre) / 4 - 1) / (g_epi_warps(pre) / 4) : 1;
}
__host__ __device__ constexpr int g_off_tail(bool pre) {
  return g_stages(pre) * G_STAGE_BYTES + G_BAR_BYTES + G_RING_BYTES + g_epi_warps(pre) * g_stage_blocks(pre) * 32 * 36;
}
static constexpr size_t G_SMEM = 1024 + g_off_tail(false);
static constexpr size_t G_SMEM_PRE = 1024 + g_off_tail(true);

struct GProb {
  CUtensorMap ta;   // A: m rows x k columns, leading dimension lda
  CUtensorMap tb;   // B: k rows x n columns, leading dimension ldb
  const uint8_t* A;
  const uint8_t* B;
  uint8_t* C;
  int lda, ldb, ldc, m, n, k;
  int ktiles;       // ceil(k / 128)
  int tm, tn;       // row blocks ceil(m / 128), column blocks ceil(n / 256)
  int tile0;        // index of this problem's first tile in the global list
  uint32_t p;
  uint32_t fdiv;    // 1 when k (p-1)^2 < 2^23: the epilogue forms each sum with one FFMA
};

// CAP problems per launch (FP_GROUP_MAX: the parameter block stays under the 32 KB limit).
template <int CAP>
struct GParamsT {
  GProb prob[CAP];
  int nprob;
  int total;        // tiles over all problems
};
using GParams = GParamsT<FP_GROUP_MAX>;
static_assert(sizeof(GParamsT<FP_GROUP_MAX>) < 32000, "kernel parameter block limit");

// Pre-tiled problems (the tensor-core share of an uneven batch, layout in fpdqt_internal.cuh):
// a stage is two plain bulk copies, no tensor map, so any row stride or alignment of the
// caller's arrays is allowed; the problem list lives in global memory and its first-tile
// indices in shared memory after the stages, so one launch takes up to F8_PRE_CAP problems.
using BProb = F8PreProb;
struct BParams {
  const BProb* prob;
  const int* tile0;
  int nprob;
  int total;
};
static_assert(G_A_BYTES == F8_BLOCK && G_B_BYTES == 2 * F8_BLOCK, "pre-tiled block size");

struct GTile {
  const GProb* pr;
  int m0, n0, mb, nb;
};

template <int CAP>
__device__ __forceinline__ GTile g_tile(const GParamsT<CAP>& g, int t) {
  int i = 0, hi = g.nprob - 1;      // the last problem whose first tile is <= t
  while (i < hi) {
    const int mid = (i + hi + 1) >> 1;
    if (g.prob[mid].tile0 <= t) i = mid;
    else hi = mid - 1;
  }
  const GProb& pr = g.prob[i];
  const int local = t - pr.tile0;
  GTile x;
  x.pr = &pr;
  x.mb = local / pr.tn;
  x.nb = local - x.mb * pr.tn;
  x.m0 = x.mb * G_BM;
  x.n0 = x.nb * G_BN;
  return x;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

// Stores one 32 x 32-byte block of C (rows r0 .. r0 + rn - 1, columns c0 .. c0 + nv - 1 of the
// block) whose bytes sit in `stg` (row r at stg + 9 r words), one warp.  16-byte stores from each
// lane's row when all 32 rows are whole and 16-byte aligned; else the lanes along the rows (one
// or two 32-byte sectors per row, not 32 rows per store), each lane writing the widest unit C's
// alignment allows: 4 bytes (8 lanes per row, 4 rows per store) when C and ldc are multiples of
// 4, 2 bytes (2 rows per store) when even, else 1.  Each group's values are read before they are
// stored, so the loads overlap; a running row pointer keeps few addresses live.
__device__ __forceinline__ void store_block(const uint32_t* stg, uint8_t* Cb, int ldc, int r0, int rn, int c0,
                                            int nv, int lane) {
  uint8_t* const dblk = Cb + (size_t)r0 * ldc + c0;
  const bool vec = lane < rn && nv >= 32 && ((((uintptr_t)(dblk + (size_t)lane * ldc)) & 15u) == 0);
  if (__all_sync(0xffffffffu, vec)) {
    const uint32_t* w = stg + lane * 9;
    uint4* d = reinterpret_cast<uint4*>(dblk + (size_t)lane * ldc);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
    return;
  }
  const uint8_t* sb = reinterpret_cast<const uint8_t*>(stg);
  const uint32_t al = (uint32_t)(((uintptr_t)Cb) | (uintptr_t)ldc);
  if ((al & 3u) == 0) {
    const int lr = lane >> 3, lc = 4 * (lane & 7);   // row in the group, first column
    const bool col_ok = lc < nv, whole = lc + 4 <= nv;
    uint8_t* d = dblk + (size_t)lr * ldc + lc;
    const size_t step = (size_t)4 * ldc;
#pragma unroll 1
    for (int h = 0; h < 8; h += 4) {
      uint32_t wv[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) wv[g] = stg[(4 * (h + g) + lr) * 9 + (lane & 7)];
#pragma unroll
      for (int g = 0; g < 4; ++g, d += step) {
        if (4 * (h + g) + lr >= rn || !col_ok) continue;
        if (whole) {
          *reinterpret_cast<uint32_t*>(d) = wv[g];
        } else {
          for (int e = 0; lc + e < nv; ++e) d[e] = (uint8_t)(wv[g] >> (8 * e));
        }
      }
    }
  } else if ((al & 1u) == 0) {
    const int lr = lane >> 4, lc = 2 * (lane & 15);
    const bool col_ok = lc < nv, whole = lc + 2 <= nv;
    uint8_t* d = dblk + (size_t)lr * ldc + lc;
    const size_t step = (size_t)2 * ldc;
#pragma unroll 1
    for (int h = 0; h < 16; h += 4) {
      uint32_t hv[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) hv[g] = *reinterpret_cast<const uint16_t*>(sb + (2 * (h + g) + lr) * 36 + lc);
#pragma unroll
      for (int g = 0; g < 4; ++g, d += step) {
        if (2 * (h + g) + lr >= rn || !col_ok) continue;
        if (whole) *reinterpret_cast<uint16_t*>(d) = (uint16_t)hv[g];
        else d[0] = (uint8_t)hv[g];
      }
    }
  } else {
    const bool col_ok = lane < nv;
    uint8_t* d = dblk + lane;
#pragma unroll 1
    for (int g8 = 0; g8 < 32; g8 += 8) {
      uint8_t b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) b[r] = sb[(g8 + r) * 36 + lane];
#pragma unroll
      for (int r = 0; r < 8; ++r, d += ldc)
        if (col_ok && g8 + r < rn) *d = b[r];
    }
  }
}

// Bit 7 of a byte of the result is set where one of the `valid` bytes at src (at most 16;
// src 16-byte aligned when valid >= 16) is >= p, with pk = 0x01010101 (128 - p): for bytes
// below 128, r + 128 - p has bit 7 set exactly when r >= p and carries into no other byte.
// Bytes past `valid` (the caller's padding, possibly unallocated) are not read.
__device__ __forceinline__ uint32_t range_bits(const uint8_t* src, int valid, uint32_t pk) {
  uint32_t w[4];
  if (valid >= 16) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t x = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * j + b < valid) x |= (uint32_t)__ldg(src + 4 * j + b) << (8 * b);
      w[j] = x;
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc |= w[j] | (w[j] + pk);
  return acc;
}

// The w-th tile of this CTA: waves of gridDim.x tiles, taken in forward order in even waves and
// in reverse order in odd ones (the tiles are sorted by inner dimension, longest first, so the
// CTAs that take the longest tile of one wave take the shortest of the next).  Every role of the
// kernel walks the same sequence; a CTA stops at its first index past the last tile (only the
// last wave can have one).
__device__ __forceinline__ int g_wave_tile(int w) {
  return w * (int)gridDim.x + ((w & 1) ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x);
}

// One tile's parameters, computed once by the producer and handed to the MMA issuer and the
// epilogue through a ring of G_RING slots in shared memory (so those roles never wait on a
// lookup in global memory between tiles).
struct TInfo {
  uint8_t* C;
  int pi;           // problem index
  int m0, n0, mb, nb;
  int m, n, ldc;
  int ktiles, klast;
  uint32_t p, fdiv, mp;   // fdiv: every sum + offset < 2^23; mp = ceil(2^32 / p)
  float mo;         // 2^23 + the offset added to every sum
};
static constexpr int G_RING = 4;
static_assert(G_RING * sizeof(TInfo) <= G_RING_BYTES, "tile parameter ring");
static_assert((2 * G_STAGES + 2 * 2 + 2 + 2 * G_RING) * 8 + 8 <= G_BAR_BYTES, "barrier area");
static_assert(G_SMEM <= 227 * 1024, "shared memory per block");

// The producer's view of a tile: its parameters and, for pre-tiled problems, the first A and B
// blocks of its row and column block.
struct TLoad {
  TInfo x;
  const uint8_t* a;
  const uint8_t* b;
};

template <int CAP>
__device__ __forceinline__ TLoad tile_load(const GParamsT<CAP>& g, const int*, const int*, int t) {
  const GTile gt = g_tile(g, t);
  const GProb& pr = *gt.pr;
  TLoad L;
  L.x.C = pr.C;
  L.x.pi = (int)(gt.pr - g.prob);
  L.x.m0 = gt.m0;
  L.x.n0 = gt.n0;
  L.x.mb = gt.mb;
  L.x.nb = gt.nb;
  L.x.m = pr.m;
  L.x.n = pr.n;
  L.x.ldc = pr.ldc;
  L.x.ktiles = pr.ktiles;
  L.x.klast = 4;
  L.x.p = pr.p;
  L.x.fdiv = pr.fdiv;
  L.x.mp = 0xFFFFFFFFu / pr.p + 1u;
  L.x.mo = 8388608.0f;
  L.a = L.b = nullptr;
  return L;
}

__device__ __forceinline__ TLoad tile_load(const BParams& g, const int* s_tile0, const int* s_tn, int t) {
  int i = 0, hi = g.nprob - 1;      // the last problem whose first tile is <= t
  while (i < hi) {
    const int mid = (i + hi + 1) >> 1;
    if (s_tile0[mid] <= t) i = mid;
    else hi = mid - 1;
  }
  const int local = t - s_tile0[i], tn = s_tn[i];
  const int mb = local / tn, nb = local - mb * tn;
  const BProb* pr = g.prob + i;
  TLoad L;
  const int ktiles = __ldg(&pr->ktiles);
  const uint32_t p = __ldg(&pr->p);
  L.x.C = pr->C;
  L.x.pi = i;
  L.x.m0 = mb * G_BM;
  L.x.n0 = nb * G_BN;
  L.x.mb = mb;
  L.x.nb = nb;
  L.x.m = __ldg(&pr->m);
  L.x.n = __ldg(&pr->n);
  L.x.ldc = __ldg(&pr->ldc);
  L.x.ktiles = ktiles;
  L.x.klast = __ldg(&pr->klast);
  L.x.p = p;
  L.x.fdiv = 1u;
  L.x.mp = 0xFFFFFFFFu / p + 1u;
  // centred operands: the sum is signed, |sum| <= k (p/2)^2; adding p T >= that makes it
  // non-negative and below 2^23 (the router guarantees it); exact: 2^23 + p T < 2^24
  L.x.mo = 8388608.0f + __ldg(&pr->off18) * 262144.0f;
  L.a = pr->At + (size_t)mb * ktiles * G_A_BYTES;
  L.b = pr->Bt + (size_t)nb * ktiles * G_B_BYTES;
  return L;
}

// PRE = false: problems in the grid-constant block, operands loaded by TMA from the caller's
// arrays.  PRE = true: pre-tiled problems from global memory (BParams), stages by bulk copies.
template <int CAP, bool PRE>
using GPar = typename std::conditional<PRE, BParams, GParamsT<CAP>>::type;

template <int CAP, bool PRE>
__global__ void __launch_bounds__(g_threads(PRE), 1) k_mm_f8g(const __grid_constant__ GPar<CAP, PRE> g, uint32_t* err) {
  constexpr int NST = g_stages(PRE), EW = g_epi_warps(PRE), NTH = g_threads(PRE);
  extern __shared__ __align__(1024) uint8_t g_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)g_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * G_STAGE_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* tfull = empty + NST;         // [2] accumulator buffer ready
  uint64_t* tempty = tfull + 2;          // [2] accumulator buffer drained
  uint64_t* drainb = tempty + 2;         // MMA completion on the abort path
  uint64_t* doneb = drainb + 1;          // every epilogue warp finished with TMEM
  uint64_t* ifull = doneb + 1;           // [G_RING] tile parameters written
  uint64_t* iempty = ifull + G_RING;     // [G_RING] tile parameters consumed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(iempty + G_RING);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  TInfo* ring = reinterpret_cast<TInfo*>(smem + NST * G_STAGE_BYTES + G_BAR_BYTES);
  uint32_t* const epi_base = reinterpret_cast<uint32_t*>(smem + NST * G_STAGE_BYTES + G_BAR_BYTES + G_RING_BYTES);
  // PRE: the problems' first tiles and column-block counts
  int* const s_tile0 = reinterpret_cast<int*>(smem + g_off_tail(PRE));
  int* const s_tn = s_tile0 + (PRE ? g.nprob : 0);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t TMEM_COLS = 512;
  if constexpr (PRE)
    for (int i = threadIdx.x; i < g.nprob; i += NTH) {
      s_tile0[i] = __ldg(g.tile0 + i);
      s_tn[i] = __ldg(&g.prob[i].tn);
    }

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);        // MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EW);      // one arrival per epilogue warp
    }
    for (int r = 0; r < G_RING; ++r) {
      mbar_init(&ifull[r], 1);        // the producer
      mbar_init(&iempty[r], EW);      // one arrival per epilogue warp
    }
    mbar_init(drainb, 1);
    mbar_init(doneb, EW);
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
    // ------------------------------------------------ producer: tile parameters, operand stages
    if (lane == 0) {
      uint32_t it = 0;              // k tiles issued by this CTA (all its tiles)
      bool stop = false;
      int t = g_wave_tile(0);
      bool have = t < g.total;
      TLoad nx;
      if (have) nx = tile_load(g, s_tile0, s_tn, t);
      for (int lt = 0; have && !stop; ++lt) {
        const TLoad cur = nx;
        // the next tile's parameters are fetched now and used one tile later
        t = g_wave_tile(lt + 1);
        have = t < g.total;
        if (have) nx = tile_load(g, s_tile0, s_tn, t);
        const int slot = lt % G_RING;
        if (lt >= G_RING && !mbar_wait(&iempty[slot], (uint32_t)((lt - G_RING) / G_RING) & 1u, abort_flag)) break;
        ring[slot] = cur.x;
        mbar_arrive(&ifull[slot]);    // release: the slot's contents are visible to the waiters
        for (int kt = 0; kt < cur.x.ktiles; ++kt, ++it) {
          const int s = (int)(it % NST);
          if (*abort_flag || !mbar_wait(&empty[s], ((it / NST) & 1u) ^ 1u, abort_flag)) {
            stop = true;
            break;
          }
          uint8_t* sa = smem + s * G_STAGE_BYTES;
          if constexpr (PRE) {
            // only what the MMAs' kept outputs read: A rows up to m (in whole 8-row groups), the
            // B rows of the K = 32 steps issued, the second 128-column half of B only if n
            // reaches it (the rest of the stage holds older bytes, which reach only accumulator
            // rows and columns the epilogue never stores)
            const uint32_t a_bytes = (uint32_t)((min(G_BM, cur.x.m - cur.x.m0) + 7) & ~7) * 128u;
            const uint32_t b_rows = kt == cur.x.ktiles - 1 ? 32u * (uint32_t)cur.x.klast : 128u;
            const uint32_t halves = cur.x.n - cur.x.n0 > 128 ? 2u : 1u;
            mbar_expect_tx(&full[s], a_bytes + halves * b_rows * 128u);
            bulk_load(sa, cur.a + (size_t)kt * G_A_BYTES, a_bytes, &full[s]);
            const uint8_t* bsrc = cur.b + (size_t)kt * G_B_BYTES;
            for (uint32_t h = 0; h < halves; ++h)
              bulk_load(sa + G_A_BYTES + h * (G_B_BYTES / 2), bsrc + h * (G_B_BYTES / 2), b_rows * 128u, &full[s]);
          } else {
            mbar_expect_tx(&full[s], G_STAGE_BYTES);
            const GProb& pr = g.prob[cur.x.pi];
            uint8_t* sb = sa + G_A_BYTES;
            tma_load_2d(sa, &pr.ta, kt * G_BK, cur.x.m0, &full[s]);
            tma_load_2d(sb, &pr.tb, cur.x.n0, kt * G_BK, &full[s]);
            tma_load_2d(sb + G_B_BYTES / 2, &pr.tb, cur.x.n0 + 128, kt * G_BK, &full[s]);
          }
        }
      }
      // every armed stage must have landed before the CTA may exit (its shared memory is reused)
      for (uint32_t j = (it > (uint32_t)NST ? it - NST : 0u); j < it; ++j)
        mbar_drain(&full[j % NST], (j / NST) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_e4m3(G_BM, G_BN, true);
      uint32_t it = 0;
      bool stop = false;
      for (int lt = 0; g_wave_tile(lt) < g.total && !stop; ++lt) {
        const int slot = lt % G_RING;
        if (!mbar_wait(&ifull[slot], (uint32_t)(lt / G_RING) & 1u, abort_flag)) break;
        const int ktiles = ring[slot].ktiles, klast = ring[slot].klast;
        const int buf = lt & 1;
        if (lt >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((lt - 2) >> 1) & 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t dtm = tmem + (uint32_t)(buf * 256);
        for (int kt = 0; kt < ktiles; ++kt, ++it) {
          const int s = (int)(it % NST);
          if (!mbar_wait(&full[s], (it / NST) & 1u, abort_flag)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint8_t* sa = smem + s * G_STAGE_BYTES;
          const uint8_t* sb = sa + G_A_BYTES;
          const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_mn_sw128(sb, G_B_BYTES / 2);
          // K = 32 per MMA: A +32 bytes in the row, B +32 rows; the last k tile of a pre-tiled
          // problem issues only the steps that hold some of its k (the rest are zero padding)
          const int nk = kt == ktiles - 1 ? klast : 4;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk < nk)
              mma_f8(dtm, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 256), idesc, (kt | kk) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!stop) mma_commit(&tfull[buf]);
      }
      if (*abort_flag) {            // every MMA issued so far completes before TMEM is freed
        mma_commit(drainb);
        mbar_drain(drainb, 0);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2 .. 2 + EW - 1)
    const int ew = warp - 2;                     // 0 .. EW - 1
    const int q = warp & 3;                      // TMEM lane quarter this warp may access
    const int cg = ew >> 2;                      // 32-column blocks cg, cg + EW / 4, ... (< 8)
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const uint32_t tid = threadIdx.x - 64;       // 0..511 over the epilogue warps
    constexpr uint32_t ET = 32 * EW;
    // this warp's stage: g_stage_blocks(PRE) blocks of 32 rows x 36 bytes
    uint32_t* const epi_stage = epi_base + ew * (g_stage_blocks(PRE) * 32 * 9);
    uint32_t bad = 0;
    for (int lt = 0; g_wave_tile(lt) < g.total; ++lt) {
      const int buf = lt & 1, slot = lt % G_RING;
      // one lane waits, the warp follows (tcgen05.ld needs all 32 lanes on the same path)
      uint32_t got = 1;
      if (lane == 0) got = mbar_wait(&ifull[slot], (uint32_t)(lt / G_RING) & 1u, abort_flag) ? 1u : 0u;
      if (!__shfl_sync(0xffffffffu, got, 0)) break;
      const TInfo x = ring[slot];
      if constexpr (!PRE) {
        const GProb& pr = g.prob[x.pi];
        {
          // range check: a residue byte r >= p (p <= 17) has bit 7 set in r | (r + 128 - p),
          // with no carry between bytes unless bit 7 of the lower byte is already set
          const uint32_t pk = 0x01010101u * (128u - pr.p);
          const uint32_t kc = (uint32_t)(pr.k + 15) >> 4;                  // 16-byte chunks per A row
          const uint32_t a_rows = (uint32_t)min(G_BM, pr.m - x.m0);
          const uint32_t a_units = a_rows * kc, a_per = (a_units + pr.tn - 1) / pr.tn;
          const uint32_t a_lo = min(a_units, (uint32_t)x.nb * a_per), a_hi = min(a_units, a_lo + a_per);
          for (uint32_t u = a_lo + tid; u < a_hi; u += ET) {
            const uint32_t r = u / kc, c = u - r * kc;
            bad |= range_bits(pr.A + (size_t)(x.m0 + r) * pr.lda + 16 * c, pr.k - 16 * (int)c, pk);
          }
          const uint32_t bc = (uint32_t)(min(G_BN, pr.n - x.n0) + 15) >> 4;  // 16-byte chunks per B row
          const uint32_t b_units = (uint32_t)pr.k * bc, b_per = (b_units + pr.tm - 1) / pr.tm;
          const uint32_t b_lo = min(b_units, (uint32_t)x.mb * b_per), b_hi = min(b_units, b_lo + b_per);
          for (uint32_t u = b_lo + tid; u < b_hi; u += ET) {
            const uint32_t r = u / bc, c = u - r * bc;
            bad |= range_bits(pr.B + (size_t)r * pr.ldb + x.n0 + 16 * c, pr.n - x.n0 - 16 * (int)c, pk);
          }
        }
      }
      got = 1;
      if (lane == 0) got = mbar_wait(&tfull[buf], (uint32_t)(lt >> 1) & 1u, abort_flag) ? 1u : 0u;
      if (!__shfl_sync(0xffffffffu, got, 0)) break;
      tc_fence_after();
      // the MMA issuer read this slot before it committed the tile: the producer may reuse it
      __syncwarp();
      if (lane == 0) mbar_arrive(&iempty[slot]);
      const int m0 = x.m0, n0 = x.n0, m = x.m, n = x.n, ldc = x.ldc;
      const uint32_t p = x.p, mp = x.mp;
      const float mo = x.mo;
      uint8_t* const Cb = x.C;
      const int row = m0 + q * 32 + lane;
      const int r0 = m0 + q * 32, rn = min(32, m - r0);
      const bool rows_in = rn > 0;               // some row of this warp's quarter is in C
      // Pre-tiled (short tiles): every block of this warp is reduced into its stage first, the
      // accumulator buffer is released, and only then are the blocks stored, so the MMAs of the
      // tile after next need not wait for the stores.  TMA problems (long tiles): each block is
      // stored as soon as it is reduced (16-byte stores straight from registers when aligned).
      int jb = 0;
      for (int cb = cg; cb < 8; cb += EW / 4, ++jb) {
        const int col0 = cb * 32;
        // a block wholly in the tile's padding (thin products) is neither read nor stored
        // (warp-uniform, so tcgen05.ld stays converged)
        if (!rows_in || n0 + col0 >= n) continue;
        // two loads of 16 columns (fewer live registers than one of 32)
        uint32_t packed[8];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t v[16];
          tmem_ld16_nowait(tmem + lane_base + (uint32_t)(buf * 256 + col0 + 16 * hh), v);
          tmem_wait();
          if (x.fdiv) {
            // Each sum is x 2^-18 with 0 <= y = x + off < 2^23 (off = p T for centred operands,
            // else 0).  One FFMA forms 2^23 + y exactly (an integer in [2^23, 2^24): its low 23
            // bits are y), and y mod p comes from an invariant-divisor multiply: floor(y / p) =
            // floor(y mp / 2^32) with mp = ceil(2^32 / p), exact for y < 2^23 and p < 2^9 (the
            // product exceeds y / p by less than 2^-9 < 1 / p).
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              uint32_t w = 0;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const uint32_t y = __float_as_uint(fmaf(__uint_as_float(v[j + u]), 262144.0f, mo)) & 0x7FFFFFu;
                w += (y - p * __umulhi(y, mp)) << (8 * u);
              }
              packed[4 * hh + (j >> 2)] = w;
            }
          } else {
            // sums below 2^24 (TMA problems with k (p-1)^2 >= 2^23): the sum is 2^-18 times the
            // integer y, so y = 2^18 x its value exactly; the same multiply-high gives y mod p
            // (its error is below 2^24 / 2^32 = 2^-8 < 1 / p for p < 2^8)
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              uint32_t w = 0;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const uint32_t y = __float2uint_rn(__uint_as_float(v[j + u]) * 262144.0f);
                w += (y - p * __umulhi(y, mp)) << (8 * u);
              }
              packed[4 * hh + (j >> 2)] = w;
            }
          }
        }
        const int c0 = n0 + col0;                   // the same for the whole warp
        if constexpr (PRE) {
          uint32_t* const stg = epi_stage + jb * (32 * 9);
#pragma unroll
          for (int j = 0; j < 8; ++j) stg[lane * 9 + j] = packed[j];
        } else {
          uint8_t* dst = Cb + (size_t)row * ldc + c0;
          const bool vec = row < m && c0 + 32 <= n && ((((uintptr_t)dst) & 15u) == 0);
          if (__all_sync(0xffffffffu, vec)) {
            reinterpret_cast<uint4*>(dst)[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            reinterpret_cast<uint4*>(dst)[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) epi_stage[lane * 9 + j] = packed[j];
            __syncwarp();
            store_block(epi_stage, Cb, ldc, r0, rn, c0, n - c0, lane);
            __syncwarp();
          }
        }
      }
      // TMEM buffer drained: the MMAs of the tile after next may start
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      if constexpr (PRE) {
        jb = 0;
        for (int cb = cg; cb < 8; cb += EW / 4, ++jb) {
          const int c0 = n0 + cb * 32;
          if (!rows_in || c0 >= n) continue;
          store_block(epi_stage + jb * (32 * 9), Cb, ldc, r0, rn, c0, n - c0, lane);
        }
        __syncwarp();                            // the stage is reused by the next tile
      }
    }
    if (bad & 0x80808080u) flag_error(err, ERR_RANGE);
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

// ---------------------------------------------------------------- host side

bool f8_direct_ok(uint32_t p, int k, const uint8_t* A, int lda, const uint8_t* B, int ldb) {
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  return p <= 17 && (uint64_t)k * pp < (1ull << 24) && (((uintptr_t)A | (uintptr_t)B) & 15u) == 0 &&
         (lda & 15) == 0 && (ldb & 15) == 0;
}

// One launch over up to CAP problems, each already validated and f8_direct_ok.
template <int CAP>
static fp_status launch_group(fp_ctx ctx, const fp_mm_problem* const* pr, int count, cudaStream_t st) {
  GParamsT<CAP> hp;    // passed by value as the kernel's (grid-constant) parameter block
  std::memset(&hp, 0, sizeof hp);
  int tile = 0;
  for (int i = 0; i < count; ++i) {
    const fp_mm_problem& x = *pr[i];
    GProb& g = hp.prob[i];
    fp_status s = make_map_ld(&g.ta, x.A, (uint64_t)x.m, (uint64_t)x.k, (uint64_t)x.lda, G_BM, 1);
    if (s != FP_OK) return s;
    s = make_map_ld(&g.tb, x.B, (uint64_t)x.k, (uint64_t)x.n, (uint64_t)x.ldb, 128, 1);
    if (s != FP_OK) return s;
    g.A = x.A;
    g.B = x.B;
    g.C = x.C;
    g.lda = x.lda;
    g.ldb = x.ldb;
    g.ldc = x.ldc;
    g.m = x.m;
    g.n = x.n;
    g.k = x.k;
    g.ktiles = (x.k + G_BK - 1) / G_BK;
    g.tm = (x.m + G_BM - 1) / G_BM;
    g.tn = (x.n + G_BN - 1) / G_BN;
    g.tile0 = tile;
    g.p = x.p;
    g.fdiv = (uint64_t)x.k * (x.p - 1) * (x.p - 1) < (1ull << 23) ? 1u : 0u;
    tile += g.tm * g.tn;
  }
  hp.nprob = count;
  hp.total = tile;
  const int grid = std::min(tile, ctx->num_sms);
  FP_CUDA(cudaFuncSetAttribute(k_mm_f8g<CAP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G_SMEM));
  FP_LAUNCH(ctx, "k_mm_f8g", st, k_mm_f8g<CAP, false><<<grid, g_threads(false), G_SMEM, st>>>(hp, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

fp_status launch_mm_f8_pretiled(fp_ctx ctx, const F8PreProb* prob, const int* tile0, int nprob, int total,
                                cudaStream_t st) {
  if (nprob <= 0 || total <= 0) return FP_OK;
  FP_CHECK(nprob <= F8_PRE_CAP, FP_EINVAL, "pre-tiled e4m3 launch: too many problems");
  const BParams hp{prob, tile0, nprob, total};
  const size_t smem = G_SMEM_PRE + 2 * sizeof(int) * (size_t)F8_PRE_CAP;
  static_assert(G_SMEM_PRE + 2 * sizeof(int) * F8_PRE_CAP <= 227 * 1024, "shared memory per block");
  const int grid = std::min(total, ctx->num_sms);
  FP_CUDA(cudaFuncSetAttribute(k_mm_f8g<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FP_LAUNCH(ctx, "k_mm_f8g_pre", st,
            k_mm_f8g<1, true><<<grid, g_threads(true), G_SMEM_PRE + 2 * sizeof(int) * (size_t)nprob, st>>>(
                hp, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

// One problem (the caller holds the context lock).
fp_status launch_mm_f8_direct(fp_ctx ctx, const fp_mm_problem& x, cudaStream_t st) {
  const fp_mm_problem* one = &x;
  return launch_group<FP_GROUP_MAX>(ctx, &one, 1, st);
}

// Problems that pass f8_direct_ok, in launches of up to FP_GROUP_MAX problems; within a launch
// the problems with the most k tiles come first so the longest tiles start earliest.
fp_status launch_mm_f8_grouped(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return launch_mm_f8_grouped_locked(ctx, pr, count, st);
}

fp_status launch_mm_f8_grouped_locked(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, cudaStream_t st) {
  std::vector<const fp_mm_problem*> v(pr, pr + count);
  std::stable_sort(v.begin(), v.end(), [](const fp_mm_problem* a, const fp_mm_problem* b) { return a->k > b->k; });
  for (size_t i = 0; i < v.size(); i += FP_GROUP_MAX) {
    const int c = (int)std::min<size_t>(FP_GROUP_MAX, v.size() - i);
    fp_status s = launch_group<FP_GROUP_MAX>(ctx, v.data() + i, c, st);
    if (s != FP_OK) return s;
  }
  return FP_OK;
}

}  // namespace fpd
