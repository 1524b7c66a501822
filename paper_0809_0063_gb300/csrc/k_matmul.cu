// Compressed modular matrix product (Sec. 7): right compression CC = A x CB with
// CB[l][j] = sum_{t<e} B[l][j e + t] Q^t (Sec. 7.4, Eq. LeftComp without the uncompress step
// since A is given uncompressed) and REDQ_e of every word of CC, plus the unpacked baselines.
//
//  k_mm_dmma   FP64 words, mma.sync m8n8k4 f64 (DMMA).  All partial sums are non-negative
//              integers below the final word < 2^52, so any accumulation order is exact.
//  k_mm_ffma   FP32 words at Qc = 2^12 (two residues), FFMA.  The inner dimension is cut in
//              chunks of kc with kc (p-1)^2 < Qc (Eq. lower per chunk) so each chunk word stays
//              below 2^24; at the end of a chunk each word's two digits are moved into a u32
//              word R at spacing 2^16, which is REDQ-reduced every 15 chunks (delayed
//              reduction, Sec. 2.2) and once at the end.  e = 1 gives the plain FFMA baseline.
//  k_mm_imma   plain baseline: u8 x u8 -> s32 mma.sync m16n8k32, exact while k (p-1)^2 < 2^31.
#include "fpdqt_internal.cuh"

namespace fpd {

// ------------------------------------------------------------------ packing / layout kernels

template <typename W>
__global__ void k_pack_cb(const uint8_t* __restrict__ B, int ldb, W* __restrict__ CB, int ldcb, int k, int n,
                          int nw, uint32_t e, uint32_t b, uint32_t p, uint32_t* err) {
  uint64_t total = (uint64_t)k * ldcb;
  uint32_t bad = 0;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    int l = (int)(idx / ldcb), j = (int)(idx % ldcb);
    uint64_t w = 0;
    if (j < nw) {
      for (int t = (int)e - 1; t >= 0; --t) {
        int col = j * (int)e + t;
        uint32_t v = col < n ? B[(size_t)l * ldb + col] : 0u;
        bad |= v >= p;
        w = (w << b) | v;
      }
    }
    CB[idx] = WordOps<W>::from_u64(w);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// dst (rows x kp, zero padded) = src (rows x cols, leading dim lds), optionally transposed:
// trans = 0: dst[r][c] = src[r][c];  trans = 1: dst[r][c] = src[c][r] (src is cols x rows).
__global__ void k_copy_pad(const uint8_t* __restrict__ src, int lds, uint8_t* __restrict__ dst, int rows,
                           int cols, int kp, int trans, uint32_t p, uint32_t* err) {
  __shared__ uint8_t tile[32][33];
  uint32_t bad = 0;
  int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int yy = ty; yy < 32; yy += 8) {
    if (!trans) {
      int r = r0 + yy, c = c0 + tx;
      uint8_t v = (r < rows && c < cols) ? src[(size_t)r * lds + c] : 0;
      bad |= v >= p;
      tile[yy][tx] = v;
    } else {
      int sr = c0 + yy, sc = r0 + tx;  // src row = dst col
      uint8_t v = (sr < cols && sc < rows) ? src[(size_t)sr * lds + sc] : 0;
      bad |= v >= p;
      tile[tx][yy] = v;
    }
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    int r = r0 + yy, c = c0 + tx;
    if (r < rows && c < kp) dst[(size_t)r * kp + c] = tile[yy][tx];
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// dst (rows x cols, leading dimension ldd) = src^T, src (cols x rows, leading dimension lds); only
// the rows x cols entries of dst are written.
__global__ void k_transpose_u8(const uint8_t* __restrict__ src, int lds, uint8_t* __restrict__ dst, int ldd,
                               int rows, int cols) {
  __shared__ uint8_t tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int yy = ty; yy < 32; yy += 8) {
    const int sr = c0 + yy, sc = r0 + tx;   // src row = dst column
    tile[tx][yy] = (sr < cols && sc < rows) ? src[(size_t)sr * lds + sc] : 0;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int r = r0 + yy, c = c0 + tx;
    if (r < rows && c < cols) dst[(size_t)r * ldd + c] = tile[yy][tx];
  }
}

// ------------------------------------------------------------------ FP64 DMMA

template <int TM, int TN>
__global__ void __launch_bounds__(128) k_mm_dmma(const uint8_t* __restrict__ A, int lda,
                                                 const double* __restrict__ CB, int ldcb,
                                                 uint8_t* __restrict__ C, int ldc, int m, int n, int k, int nw,
                                                 uint32_t e, RedqParams P, uint32_t* err) {
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector corr;
  corr.init(P, ptab);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.y * 2 + (warp >> 1)) * (8 * TM);
  const int c0 = (blockIdx.x * 2 + (warp & 1)) * (8 * TN);
  double acc[TM][TN][2];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  uint32_t bad = 0;
  for (int k0 = 0; k0 < k; k0 += 4) {
    const int kk = k0 + t;
    double a[TM], bf[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int row = r0 + 8 * i + g;
      uint32_t v = (row < m && kk < k) ? A[(size_t)row * lda + kk] : 0u;
      bad |= v >= P.p;
      a[i] = (double)v;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int col = c0 + 8 * j + g;
      bf[j] = (col < nw && kk < k) ? CB[(size_t)kk * ldcb + col] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                     : "d"(a[i]), "d"(bf[j]));
  }
  if (bad) flag_error(err, ERR_RANGE);
  // epilogue: stage the CTA's words in shared memory, then REDQ_e of every word in a rolled
  // loop (all lanes of each warp take part in every lookup)
  constexpr int CM = 16 * TM, CN = 16 * TN;
  __shared__ double sw[CM * CN];
  const int lr0 = (warp >> 1) * (8 * TM), lc0 = (warp & 1) * (8 * TN);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) sw[(lr0 + 8 * i + g) * CN + lc0 + 8 * j + 2 * t + h] = acc[i][j][h];
  __syncthreads();
  const int R0 = blockIdx.y * CM, Cw0 = blockIdx.x * CN;
#pragma unroll 1
  for (int idx = threadIdx.x; idx < CM * CN; idx += blockDim.x) {
    const int row = R0 + idx / CN, col = Cw0 + idx % CN;
    const bool own = row < m && col < nw;
    uint8_t* dst = C + (size_t)(own ? row : 0) * ldc;
    redq_word<double>(sw[idx], P, corr, [&](uint32_t tt, uint32_t mu) {
      int cc = col * (int)e + (int)tt;
      if (own && cc < n) dst[cc] = (uint8_t)mu;
    });
  }
}

// ------------------------------------------------------------------ CMM: middle product (Sec. 7.1)
//
// A m x k packed along rows, d+1 consecutive entries of the inner dimension per FP64 word and
// REVERSED (entry j(d+1)+i at q^(d-i)); B k x n packed along columns, FORWARD (entry j(d+1)+i at
// q^i).  The word product of a row block and a column block then holds the block's dot product
// as its digit of q^d, and summing the word products over the kw = ceil(k/(d+1)) blocks sums the
// dot products there.  q = 2^b > k (p-1)^2 keeps every digit below q, and (2d+1) b <= 52 keeps
// every word product and partial sum an exact integer below 2^52, so the digit is read off
// exactly: C_ij = ((w >> d b) & (q - 1)) mod p.

// CA[r][j] = sum_i A[r][j(d+1)+i] q^(d-i)  (m x kw); CB[j][c] = sum_i B[j(d+1)+i][c] q^i  (kw x n).
__global__ void k_cmm_pack(const uint8_t* __restrict__ A, int lda, const uint8_t* __restrict__ B, int ldb,
                           double* __restrict__ CA, double* __restrict__ CB, int m, int n, int k, int kw, uint32_t d1,
                           uint32_t b, uint32_t p, uint32_t* err) {
  const uint64_t na = (uint64_t)m * kw, total = na + (uint64_t)kw * n;
  uint32_t bad = 0;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t w = 0;
    if (idx < na) {
      const int r = (int)(idx / kw), j = (int)(idx % kw);
      for (uint32_t i = 0; i < d1; ++i) {          // Horner from entry 0: reversed order
        const int l = j * (int)d1 + (int)i;
        const uint32_t v = l < k ? A[(size_t)r * lda + l] : 0u;
        bad |= v >= p;
        w = (w << b) | v;
      }
      CA[idx] = (double)w;
    } else {
      const uint64_t i2 = idx - na;
      const int j = (int)(i2 / n), c = (int)(i2 % n);
      for (int i = (int)d1 - 1; i >= 0; --i) {     // forward: entry 0 lowest
        const int l = j * (int)d1 + i;
        const uint32_t v = l < k ? B[(size_t)l * ldb + c] : 0u;
        bad |= v >= p;
        w = (w << b) | v;
      }
      CB[i2] = (double)w;
    }
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// C = (CA x CB) digit d mod p on DMMA (mma.sync m8n8k4 f64), the same warp tiling as k_mm_dmma.
template <int TM, int TN>
__global__ void __launch_bounds__(128) k_mm_cmm(const double* __restrict__ CA, const double* __restrict__ CB,
                                                uint8_t* __restrict__ C, int ldc, int m, int n, int kw,
                                                uint32_t shift, uint64_t qmask, DivP dv, uint32_t p) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.y * 2 + (warp >> 1)) * (8 * TM);
  const int c0 = (blockIdx.x * 2 + (warp & 1)) * (8 * TN);
  double acc[TM][TN][2];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  for (int k0 = 0; k0 < kw; k0 += 4) {
    const int kk = k0 + t;
    double a[TM], bf[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = r0 + 8 * i + g;
      a[i] = (row < m && kk < kw) ? CA[(size_t)row * kw + kk] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int col = c0 + 8 * j + g;
      bf[j] = (col < n && kk < kw) ? CB[(size_t)kk * n + col] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                     : "d"(a[i]), "d"(bf[j]));
  }
  // accumulator (i, j, h) holds row r0 + 8i + g, column c0 + 8j + 2t + h
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = r0 + 8 * i + g, col = c0 + 8 * j + 2 * t + h;
        if (row < m && col < n) {
          const uint64_t w = (uint64_t)acc[i][j][h];        // exact integer < 2^52
          C[(size_t)row * ldc + col] = (uint8_t)modp32((uint32_t)((w >> shift) & qmask), dv, p);
        }
      }
}

// ------------------------------------------------------------------ FP32 FFMA (packed e=2 / plain e=1)

static constexpr int FF_BM = 128, FF_BN = 128, FF_BK = 8;
static constexpr size_t FF_DYN_SMEM = FF_BM * FF_BN * sizeof(uint32_t);
extern __shared__ __align__(16) uint8_t ffma_dyn_smem[];

template <int E>
__global__ void __launch_bounds__(256, 1) k_mm_ffma(const uint8_t* __restrict__ A, int lda,
                                                    const float* __restrict__ CB, int ldcb,
                                                    uint8_t* __restrict__ C, int ldc, int m, int n, int k, int nw,
                                                    int chunk_tiles, RedqParams Pr,
                                                    uint32_t* err) {
  // Pr: REDQ of the running u32 word (q = 2^16, E digits) used both for the periodic
  // re-reduction and for the final residues.
  __shared__ __align__(16) float As[2][FF_BK][FF_BM];
  __shared__ __align__(16) float Bs[2][FF_BK][FF_BN];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, Pr);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * FF_BM, n0 = blockIdx.x * FF_BN;
  Corrector corr;
  corr.init(Pr, ptab);

  float acc[8][8];
  uint32_t R[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) { acc[i][j] = 0.f; R[i][j] = 0u; }

  // global -> register staging indices
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;      // 128 rows x 8 k
  const int b_k = tid >> 5, b_col = (tid & 31) * 4;     // 8 k x 128 words
  uint32_t bad = 0;
  const int ktiles = (k + FF_BK - 1) / FF_BK;

  auto load_tile = [&](int kt, float (&ra)[4], float4& rb) {
    const int kbase = kt * FF_BK;
    const int row = m0 + a_row;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int kk = kbase + a_k + q;
      uint32_t v = (row < m && kk < k) ? A[(size_t)row * lda + kk] : 0u;
      bad |= v >= Pr.p;
      ra[q] = (float)v;
    }
    int kk = kbase + b_k, col = n0 + b_col;
    if (kk < k && col < ldcb) rb = *reinterpret_cast<const float4*>(CB + (size_t)kk * ldcb + col);
    else rb = make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store_tile = [&](int buf, const float (&ra)[4], const float4& rb) {
#pragma unroll
    for (int q = 0; q < 4; ++q) As[buf][a_k + q][a_row] = ra[q];
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_col]) = rb;
  };

  // fold: move the chunk accumulator's E digits (spacing 2^12) into R (spacing 2^16)
  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t vi = __float2uint_rz(acc[i][j]);
        if (E == 2) R[i][j] += vi + (vi >> 12) * (65536u - 4096u);
        else R[i][j] += vi;
        acc[i][j] = 0.f;
      }
  };
  // periodic delayed reduction of R: each 16-bit digit is replaced by its residue mod p
  auto rereduce = [&]() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t v = R[i][j];
        if (E == 2) R[i][j] = modp32(v & 0xffffu, Pr.dv, Pr.p) | (modp32(v >> 16, Pr.dv, Pr.p) << 16);
        else R[i][j] = modp32(v, Pr.dv, Pr.p);
      }
  };

  float ra[4];
  float4 rb;
  load_tile(0, ra, rb);
  store_tile(0, ra, rb);
  __syncthreads();
  int folds = 0;
  int in_chunk = 0;
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) load_tile(kt + 1, ra, rb);
#pragma unroll
    for (int kk = 0; kk < FF_BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (++in_chunk == chunk_tiles) {
      fold();
      in_chunk = 0;
      if (++folds == (E == 2 ? 15 : 255)) {
        rereduce();
        folds = 0;
      }
    }
    if (kt + 1 < ktiles) {
      store_tile(buf ^ 1, ra, rb);
    }
    __syncthreads();
  }
  if (in_chunk) fold();
  if (bad) flag_error(err, ERR_RANGE);
  // final REDQ_E of R: stage the CTA tile of words in shared memory (reusing the operand
  // tiles' space is not enough, so a dedicated dynamic buffer), then a rolled loop in which
  // consecutive threads take consecutive words of a row (coalesced stores of E residues)
  uint32_t* sR = reinterpret_cast<uint32_t*>(ffma_dyn_smem);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int rl = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cl = j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4);
      sR[rl * FF_BN + cl] = R[i][j];
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int idx = tid; idx < FF_BM * FF_BN; idx += 256) {
    const int row = m0 + idx / FF_BN, col = n0 + idx % FF_BN;
    const bool own = row < m && col < nw;
    uint8_t* dst = C + (size_t)(own ? row : 0) * ldc;
    redq_word<uint32_t>(sR[idx], Pr, corr, [&](uint32_t tt, uint32_t mu) {
      int cc = col * E + (int)tt;
      if (own && cc < n) dst[cc] = (uint8_t)mu;
    });
  }
}

// ------------------------------------------------------------------ u8 IMMA (plain)

static constexpr int IM_BM = 128, IM_BN = 128, IM_BK = 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// byte offset of 16-byte chunk c (0..3) of row r in a 64-byte-row tile, XOR-swizzled so that
// ldmatrix's 8 rows at the same chunk hit distinct banks
__device__ __forceinline__ int im_off(int r, int c) { return r * 64 + ((c ^ ((r >> 1) & 3)) << 4); }

// A2: m x kp (K contiguous), Bt: n x kp (K contiguous), both zero padded, kp % 64 == 0.
__global__ void __launch_bounds__(256) k_mm_imma(const uint8_t* __restrict__ A2, const uint8_t* __restrict__ Bt,
                                                 int kp, uint8_t* __restrict__ C, int ldc, int m, int n,
                                                 uint32_t p, DivP dv) {
  __shared__ __align__(128) uint8_t sA[2][IM_BM * IM_BK];
  __shared__ __align__(128) uint8_t sB[2][IM_BN * IM_BK];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;       // 2 x 4 warps, warp tile 64 x 32
  const int m0 = blockIdx.y * IM_BM, n0 = blockIdx.x * IM_BN;
  int acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0;

  const int ktiles = kp / IM_BK;
  auto issue = [&](int kt, int buf) {
    // 128 rows x 4 chunks for A and for B: 512 + 512 chunks, 4 per thread
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int id = tid + q * 256;
      int r = id >> 2, c = id & 3;
      int gr = m0 + r;
      const uint8_t* src = A2 + (size_t)(gr < m ? gr : 0) * kp + kt * IM_BK + c * 16;
      if (gr < m) cp_async16(&sA[buf][im_off(r, c)], src);
      else *reinterpret_cast<uint4*>(&sA[buf][im_off(r, c)]) = make_uint4(0, 0, 0, 0);
      int gn = n0 + r;
      const uint8_t* srcb = Bt + (size_t)(gn < n ? gn : 0) * kp + kt * IM_BK + c * 16;
      if (gn < n) cp_async16(&sB[buf][im_off(r, c)], srcb);
      else *reinterpret_cast<uint4*>(&sB[buf][im_off(r, c)]) = make_uint4(0, 0, 0, 0);
    }
    cp_async_commit();
  };
  issue(0, 0);
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) {
      issue(kt + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {  // two k32 steps per 64-byte tile
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        // lanes 0-7 rows 0-7 chunk 2ks, 8-15 rows 8-15 chunk 2ks, 16-23 rows 0-7 chunk 2ks+1, ...
        int r = wm * 64 + i * 16 + (lane & 15);
        int c = ks * 2 + (lane >> 4);
        uint32_t addr = smem_u32(&sA[buf][im_off(r, c)]);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(af[i][0]), "=r"(af[i][1]), "=r"(af[i][2]), "=r"(af[i][3])
                     : "r"(addr));
      }
#pragma unroll
      for (int j2 = 0; j2 < 2; ++j2) {
        // two n8 blocks per ldmatrix.x4: lanes 0-7 n rows 0-7 chunk 2ks, 8-15 same rows chunk
        // 2ks+1, 16-23 n rows 8-15 chunk 2ks, 24-31 n rows 8-15 chunk 2ks+1
        int r = wn * 32 + j2 * 16 + (lane & 7) + ((lane >> 4) << 3);
        int c = ks * 2 + ((lane >> 3) & 1);
        uint32_t addr = smem_u32(&sB[buf][im_off(r, c)]);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(bfr[2 * j2][0]), "=r"(bfr[2 * j2][1]), "=r"(bfr[2 * j2 + 1][0]),
                       "=r"(bfr[2 * j2 + 1][1])
                     : "r"(addr));
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+r"(acc[i][j][0]), "+r"(acc[i][j][1]), "+r"(acc[i][j][2]), "+r"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                "r"(bfr[j][1]));
    }
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int row = m0 + wm * 64 + i * 16 + g + ((q >> 1) << 3);
        int col = n0 + wn * 32 + j * 8 + 2 * t + (q & 1);
        if (row < m && col < n) C[(size_t)row * ldc + col] = (uint8_t)modp32((uint32_t)acc[i][j][q], dv, p);
      }
}

// ------------------------------------------------------------------ launchers

fp_status mm_choose(uint32_t p, uint64_t kdim, uint32_t algo, uint32_t* b, uint32_t* e, uint32_t* chunk);
fp_status launch_mm_tc(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                       const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st);

template <typename W>
static fp_status pack_cb_t(fp_ctx ctx, uint32_t p, int k, int n, const uint8_t* B, int ldb, uint32_t b,
                           uint32_t e, W* CB, int ldcb, cudaStream_t st) {
  int nw = (n + (int)e - 1) / (int)e;
  uint64_t total = (uint64_t)k * ldcb;
  int grid = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->num_sms * 16);
  FP_LAUNCH(ctx, "k_pack_cb", st, k_pack_cb<W><<<grid, 256, 0, st>>>(B, ldb, CB, ldcb, k, n, nw, e, b, p, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

fp_status launch_pack_cb(fp_ctx ctx, uint32_t p, int k, int n, const uint8_t* B, int ldb, uint32_t b,
                         uint32_t e, uint32_t word, void* CB, cudaStream_t st) {
  int nw = (n + (int)e - 1) / (int)e;
  switch (word) {
    case FP_WORD_F64: return pack_cb_t<double>(ctx, p, k, n, B, ldb, b, e, (double*)CB, nw, st);
    case FP_WORD_F32: return pack_cb_t<float>(ctx, p, k, n, B, ldb, b, e, (float*)CB, nw, st);
    default: return pack_cb_t<uint64_t>(ctx, p, k, n, B, ldb, b, e, (uint64_t*)CB, nw, st);
  }
}

static fp_status mm_dmma(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                         const uint8_t* B, int ldb, uint8_t* C, int ldc, bool plain, cudaStream_t st) {
  uint32_t b, e, chunk;
  fp_status s = mm_choose(p, (uint64_t)k, plain ? FP_MM_PLAIN_F64 : FP_MM_RIGHT_F64, &b, &e, &chunk);
  if (s != FP_OK) return s;
  int nw = (n + (int)e - 1) / (int)e;
  s = ensure_scratch(ctx, (size_t)k * nw * sizeof(double), 0, st);
  if (s != FP_OK) return s;
  double* CB = (double*)ctx->scratch;
  s = pack_cb_t<double>(ctx, p, k, n, B, ldb, b, e, CB, nw, st);
  if (s != FP_OK) return s;
  RedqParams P = make_redq(p, b, e);
  // warp tile 32x32 words when that gives >= 2 warps per SM sub-partition, else 16x16
  uint64_t warps_big = (uint64_t)((m + 31) / 32) * ((nw + 31) / 32);
  if (warps_big >= (uint64_t)ctx->num_sms * 8) {
    dim3 grid((nw + 63) / 64, (m + 63) / 64);
    FP_LAUNCH(ctx, "k_mm_dmma", st, k_mm_dmma<4, 4><<<grid, 128, 0, st>>>(A, lda, CB, nw, C, ldc, m, n, k, nw, e, P, ctx->d_err));
  } else {
    dim3 grid((nw + 31) / 32, (m + 31) / 32);
    FP_LAUNCH(ctx, "k_mm_dmma", st, k_mm_dmma<2, 2><<<grid, 128, 0, st>>>(A, lda, CB, nw, C, ldc, m, n, k, nw, e, P, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

static fp_status mm_ffma(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                         const uint8_t* B, int ldb, uint8_t* C, int ldc, bool plain, cudaStream_t st) {
  uint32_t E, chunk, bq;
  if (plain) {
    uint64_t pp = (uint64_t)(p - 1) * (p - 1);
    uint64_t kc = pp ? ((1ull << 24) - 1) / pp : (1ull << 24);
    kc &= ~7ull;
    FP_CHECK(kc >= 8, FP_EBOUND, "PLAIN_F32 needs (p-1)^2 < 2^21");
    E = 1;
    bq = 16;
    chunk = (uint32_t)std::min<uint64_t>(kc, 1u << 30);
  } else {
    fp_status s = mm_choose(p, (uint64_t)k, FP_MM_RIGHT_F32, &bq, &E, &chunk);
    if (s != FP_OK) return s;
  }
  int nw = (n + (int)E - 1) / (int)E;
  int ldcb = (nw + 3) & ~3;
  fp_status s = ensure_scratch(ctx, (size_t)k * ldcb * sizeof(float), 0, st);
  if (s != FP_OK) return s;
  float* CB = (float*)ctx->scratch;
  s = pack_cb_t<float>(ctx, p, k, n, B, ldb, 12, E, CB, ldcb, st);
  if (s != FP_OK) return s;
  int chunk_tiles = (int)(chunk / FF_BK);
  if (chunk_tiles < 1) chunk_tiles = 1;
  RedqParams Pr = make_redq(p, 16, E);
  dim3 grid((nw + FF_BN - 1) / FF_BN, (m + FF_BM - 1) / FF_BM);
  FP_CUDA(cudaFuncSetAttribute(k_mm_ffma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FF_DYN_SMEM));
  FP_CUDA(cudaFuncSetAttribute(k_mm_ffma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FF_DYN_SMEM));
  if (E == 2)
    FP_LAUNCH(ctx, "k_mm_ffma", st, k_mm_ffma<2><<<grid, 256, FF_DYN_SMEM, st>>>(A, lda, CB, ldcb, C, ldc, m, n, k, nw, chunk_tiles, Pr, ctx->d_err));
  else
    FP_LAUNCH(ctx, "k_mm_ffma", st, k_mm_ffma<1><<<grid, 256, FF_DYN_SMEM, st>>>(A, lda, CB, ldcb, C, ldc, m, n, k, nw, chunk_tiles, Pr, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

static fp_status mm_imma(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                         const uint8_t* B, int ldb, uint8_t* C, int ldc, cudaStream_t st) {
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  FP_CHECK((uint64_t)k * pp < (1ull << 31), FP_EBOUND, "PLAIN_I8 needs k (p-1)^2 < 2^31");
  int kp = (k + IM_BK - 1) / IM_BK * IM_BK;
  size_t abytes = (size_t)m * kp, bbytes = (size_t)n * kp;
  fp_status s = ensure_scratch(ctx, abytes + bbytes, 0, st);
  if (s != FP_OK) return s;
  uint8_t* A2 = (uint8_t*)ctx->scratch;
  uint8_t* Bt = A2 + abytes;
  dim3 ga((kp + 31) / 32, (m + 31) / 32);
  FP_LAUNCH(ctx, "k_copy_pad", st, k_copy_pad<<<ga, 256, 0, st>>>(A, lda, A2, m, k, kp, 0, p, ctx->d_err));
  dim3 gb((kp + 31) / 32, (n + 31) / 32);
  FP_LAUNCH(ctx, "k_copy_pad", st, k_copy_pad<<<gb, 256, 0, st>>>(B, ldb, Bt, n, k, kp, 1, p, ctx->d_err));
  dim3 grid((n + IM_BN - 1) / IM_BN, (m + IM_BM - 1) / IM_BM);
  FP_LAUNCH(ctx, "k_mm_imma", st, k_mm_imma<<<grid, 256, 0, st>>>(A2, Bt, kp, C, ldc, m, n, p, make_divp(p)));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

// The middle-product parameters: b with 2^b > k (p-1)^2 (strict, Eq. lower), d + 1 entries per
// word, d the largest with (2d+1) b <= 52 (every word product and sum an exact FP64 integer).
static fp_status cmm_choose(uint32_t p, uint64_t k, uint32_t* b_out, uint32_t* d1_out) {
  const uint64_t D = k * (uint64_t)(p - 1) * (p - 1);
  uint32_t b = 1;
  while (b < 64 && (1ull << b) <= D) ++b;
  const uint32_t d = b <= 52 ? (52 / b - 1) / 2 : 0;
  FP_CHECK(d >= 1, FP_EBOUND, "CMM_F64 needs k (p-1)^2 < 2^17 (k=%llu p=%u)", (unsigned long long)k, p);
  *b_out = b;
  *d1_out = d + 1;
  return FP_OK;
}

static fp_status mm_cmm(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                        int ldb, uint8_t* C, int ldc, cudaStream_t st) {
  uint32_t b, d1;
  fp_status s = cmm_choose(p, (uint64_t)k, &b, &d1);
  if (s != FP_OK) return s;
  const int kw = (k + (int)d1 - 1) / (int)d1;
  const size_t ca = (((size_t)m * kw * sizeof(double)) + 255) & ~(size_t)255;
  s = ensure_scratch(ctx, ca + (size_t)kw * n * sizeof(double), 0, st);
  if (s != FP_OK) return s;
  double* CA = (double*)ctx->scratch;
  double* CB = (double*)((uint8_t*)ctx->scratch + ca);
  const uint64_t total = (uint64_t)m * kw + (uint64_t)kw * n;
  const int pg = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->num_sms * 16);
  FP_LAUNCH(ctx, "k_cmm_pack", st, k_cmm_pack<<<pg, 256, 0, st>>>(A, lda, B, ldb, CA, CB, m, n, k, kw, d1, b, p,
                                                                  ctx->d_err));
  const uint32_t shift = (d1 - 1) * b;
  const uint64_t qmask = (1ull << b) - 1;
  const uint64_t warps_big = (uint64_t)((m + 31) / 32) * ((n + 31) / 32);
  if (warps_big >= (uint64_t)ctx->num_sms * 8) {
    dim3 grid((n + 63) / 64, (m + 63) / 64);
    FP_LAUNCH(ctx, "k_mm_cmm", st, k_mm_cmm<4, 4><<<grid, 128, 0, st>>>(CA, CB, C, ldc, m, n, kw, shift, qmask,
                                                                        make_divp(p), p));
  } else {
    dim3 grid((n + 31) / 32, (m + 31) / 32);
    FP_LAUNCH(ctx, "k_mm_cmm", st, k_mm_cmm<2, 2><<<grid, 128, 0, st>>>(CA, CB, C, ldc, m, n, kw, shift, qmask,
                                                                        make_divp(p), p));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

// Left compression (Sec. 7.4) by transposition: (A B)^T = B^T A^T, whose right compression packs
// consecutive columns of A^T, i.e. consecutive rows of A, into one word.  A^T (k x m) and B^T
// (n x k) are written to context scratch slot 1 (range-checked on the way), the right-compressed
// product (which packs its words in slot 0) computes C^T (n x m) there, and one transpose writes
// the m x n entries of C.
static fp_status mm_left(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                         int ldb, uint8_t* C, int ldc, bool f64, cudaStream_t st) {
  uint32_t b, e, c;
  fp_status s = mm_choose(p, (uint64_t)k, f64 ? FP_MM_RIGHT_F64 : FP_MM_RIGHT_F32, &b, &e, &c);
  if (s != FP_OK) return s;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t at = al((size_t)k * m), bt = al((size_t)n * k), ct = al((size_t)n * m);
  s = ensure_scratch(ctx, at + bt + ct, 1, st);
  if (s != FP_OK) return s;
  uint8_t* At = (uint8_t*)ctx->scratch2;
  uint8_t* Bt = At + at;
  uint8_t* Ct = Bt + bt;
  dim3 ga((m + 31) / 32, (k + 31) / 32);
  FP_LAUNCH(ctx, "k_copy_pad", st, k_copy_pad<<<ga, 256, 0, st>>>(A, lda, At, k, m, m, 1, p, ctx->d_err));
  dim3 gb((k + 31) / 32, (n + 31) / 32);
  FP_LAUNCH(ctx, "k_copy_pad", st, k_copy_pad<<<gb, 256, 0, st>>>(B, ldb, Bt, n, k, k, 1, p, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  s = f64 ? mm_dmma(ctx, p, n, m, k, Bt, k, At, m, Ct, m, false, st)
          : mm_ffma(ctx, p, n, m, k, Bt, k, At, m, Ct, m, false, st);
  if (s != FP_OK) return s;
  dim3 gc((n + 31) / 32, (m + 31) / 32);
  FP_LAUNCH(ctx, "k_transpose_u8", st, k_transpose_u8<<<gc, 256, 0, st>>>(Ct, m, C, ldc, m, n));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

static fp_status run_algo(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                          const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st) {
  switch (algo) {
    case FP_MM_FULL_F64: return mm_full(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, st);
    case FP_MM_SPLIT_F64: return mm_split(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, st);
    case FP_MM_CMM_F64: return mm_cmm(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, st);
    case FP_MM_LEFT_F64: return mm_left(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, true, st);
    case FP_MM_LEFT_F32: return mm_left(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, false, st);
    case FP_MM_RIGHT_F64: return mm_dmma(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, false, st);
    case FP_MM_PLAIN_F64: return mm_dmma(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, true, st);
    case FP_MM_RIGHT_F32: return mm_ffma(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, false, st);
    case FP_MM_PLAIN_F32: return mm_ffma(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, true, st);
    case FP_MM_PLAIN_I8: return mm_imma(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, st);
    case FP_MM_PLAIN_TC:
    case FP_MM_PLAIN_F8:
    case FP_MM_RIGHT_TC: return launch_mm_tc(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, algo, st);
    default:
      set_error("fp_matmul: algorithm %d not available", algo);
      return FP_EUNSUPPORTED;
  }
}

// Exact candidates for (p, k), fastest first by the fixed rule measured on GB300: packed
// tensor-core words (p <= 3, large products), plain tensor cores, u8 tensor cores, packed FP32
// words, packed FP64 words (always valid for k (p-1)^2 < 2^52).
// The exactness rule of a forced algorithm, checked on the host (the same conditions the
// launch paths enforce), so a group can be refused before anything is enqueued.
fp_status mm_bound_check(uint32_t p, int k, int algo) {
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  uint32_t b, e, c;
  switch (algo) {
    case FP_MM_RIGHT_F64:
    case FP_MM_RIGHT_F32: return mm_choose(p, (uint64_t)k, (uint32_t)algo, &b, &e, &c);
    case FP_MM_LEFT_F64: return mm_choose(p, (uint64_t)k, FP_MM_RIGHT_F64, &b, &e, &c);
    case FP_MM_CMM_F64: return cmm_choose(p, (uint64_t)k, &b, &e);
    case FP_MM_FULL_F64: {
      uint32_t d1, piece;
      return full_choose(p, (uint64_t)k, &b, &d1, &e, &piece);
    }
    case FP_MM_SPLIT_F64: return split_choose(p, (uint64_t)k, &b, &e, &c);
    case FP_MM_LEFT_F32: return mm_choose(p, (uint64_t)k, FP_MM_RIGHT_F32, &b, &e, &c);
    case FP_MM_PLAIN_I8:
      FP_CHECK((uint64_t)k * pp < (1ull << 31), FP_EBOUND, "PLAIN_I8 needs k (p-1)^2 < 2^31");
      return FP_OK;
    case FP_MM_PLAIN_TC:
      FP_CHECK((uint64_t)k * pp < (1ull << 24), FP_EBOUND, "PLAIN_TC needs k (p-1)^2 < 2^24");
      return FP_OK;
    case FP_MM_PLAIN_F8:
      FP_CHECK(p <= 17 && (uint64_t)k * pp < (1ull << 24), FP_EBOUND, "PLAIN_F8 needs p <= 17, k (p-1)^2 < 2^24");
      return FP_OK;
    case FP_MM_RIGHT_TC:
      FP_CHECK(f16p_ok(p, k), FP_EBOUND, "RIGHT_TC needs p <= 3 with k <= 32767, or p in {5, 7}");
      return FP_OK;
    default: return FP_OK;   // AUTO, PLAIN_F64, PLAIN_F32: every p <= 251, k <= 2^20
  }
}

static int candidates(uint32_t p, int m, int n, int k, int* out) {
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  int c = 0;
  bool big = (uint64_t)m * n >= (uint64_t)2048 * 2048;
  if (p <= 17 && (uint64_t)k * pp < (1ull << 24)) out[c++] = FP_MM_PLAIN_F8;
  if (p <= 3 && k <= 32767 && big) out[c++] = FP_MM_RIGHT_TC;
  if ((uint64_t)k * pp < (1ull << 24)) out[c++] = FP_MM_PLAIN_TC;
  if (p <= 3 && k <= 32767 && !big) out[c++] = FP_MM_RIGHT_TC;
  if ((uint64_t)k * pp < (1ull << 31)) out[c++] = FP_MM_PLAIN_I8;
  if (pp <= 511) out[c++] = FP_MM_RIGHT_F32;
  out[c++] = FP_MM_RIGHT_F64;
  return c;
}

static uint64_t tune_key(uint32_t p, int m, int n, int k) {
  auto lg = [](int x) { uint64_t b = 0; while ((1 << b) < x) ++b; return b; };
  return ((uint64_t)p << 32) | (lg(m) << 20) | (lg(n) << 10) | lg(k);
}

fp_status launch_matmul(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                        const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);  // scratch is shared by calls on this context
  if (algo != FP_MM_AUTO) return run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, algo, st);
  // e4m3 operands (the caller's bytes, or a padded copy of them): fastest measured at every
  // size wherever its exactness rule holds
  if (p <= 17 && (uint64_t)k * (p - 1) * (p - 1) < (1ull << 24))
    return run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, FP_MM_PLAIN_F8, st);
  int cand[8];
  const int nc = candidates(p, m, n, k, cand);
  const uint64_t key = tune_key(p, m, n, k);
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, it->second, st);
  // no timing with tuning off or inside a stream capture (it synchronises): the fixed rule
  if (!ctx->autotune || nc == 1 || stream_capturing(st))
    return run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, cand[0], st);
  // autotune: time each exact candidate once (all write the same C), keep the fastest;
  // FP64 words are only timed when nothing faster is valid
  cudaEvent_t e0, e1;
  FP_CUDA(cudaEventCreate(&e0));
  const cudaError_t ee = cudaEventCreate(&e1);
  if (ee != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ee, "cudaEventCreate");
  }
  int best = cand[0];
  float best_ms = 1e30f;
  for (int i = 0; i < nc; ++i) {
    if (cand[i] == FP_MM_RIGHT_F64 && i > 0) break;
    // warm (first-use costs such as scratch growth are not the kernel's)
    fp_status s = run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, cand[i], st);
    if (s != FP_OK) continue;
    cudaEventRecord(e0, st);
    s = run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, cand[i], st);
    cudaEventRecord(e1, st);
    if (s != FP_OK) continue;
    float ms = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    if (ms < best_ms) { best_ms = ms; best = cand[i]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune[key] = best;
  return run_algo(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, best, st);
}

}  // namespace fpd

extern "C" fp_status fp_ctx_autotune(fp_ctx ctx, int enable) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_ctx_autotune: ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->autotune = enable ? 1 : 0;
  if (enable == 2) ctx->tune.clear();
  return FP_OK;
}

extern "C" fp_status fp_ctx_autotune_choice(fp_ctx ctx, uint32_t p, int m, int n, int k, int* algo) {
  FP_CHECK(ctx && algo, FP_EINVAL, "fp_ctx_autotune_choice: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->tune.find(fpd::tune_key(p, m, n, k));
  *algo = it == ctx->tune.end() ? -1 : it->second;
  return FP_OK;
}
