// Full compression (Sec. 7.5) and right compression with the inner dimension split into pieces
// (Sec. 7.6, the 2049 = 1024 + 1025 remark after Table comprange), both on FP64 words and the
// FP64 tensor cores (DMMA, mma.sync m8n8k4 f64).
//
// Full compression packs dq1 = d_q + 1 consecutive rows of A into one word at Q = 2^b and
// dt1 = d_theta + 1 consecutive columns of B into one word at Theta = Q^s, s = dq1 (the
// smallest Theta Eq. qtheta allows).  The exact integer product of the packed operands,
// summed over the inner dimension, holds C[r dq1 + i][c dt1 + j] as its base-Q digit i + s j
// (every digit is below Q by Eq. lower, so no digit carries); REDQ over the ndig = s (dt1-1) + dq1
// digits gives them mod p.  Right compression is the case dq1 = s = 1, dt1 = e.
//
// Splitting: when the inner dimension k is too long for the packing to stay exact, it is cut
// into pieces of at most `piece` entries that each satisfy Eq. lower at the chosen Q.  At the
// end of a piece every accumulator word is an exact integer whose digits are bit fields (Q is a
// power of two and each digit is below Q); they are added into a 64-bit word R whose fields are
// w = floor(64 / ndig) bits wide, the accumulator restarts at zero, and every `refold` pieces
// (before any field could reach 2^w) R is replaced by the residues of its fields through REDQ at
// q = 2^w.  The last REDQ of R gives C.  The sum of the pieces' digits is the digit of the
// unsplit product, so C is the same; the pieces add the modular reductions the paper mentions.
//
// The packed words are formed once by integer shifts in a packing pass (B always, A for full
// compression) and read by the DMMA loop as doubles: FP64 conversions or FMAs in the loop
// would take the same slow FP64 pipe as the DMMA instructions themselves.
#include <cmath>

#include "fpdqt_internal.cuh"

namespace fpd {

struct FsParams {
  int m, n, k;           // C is m x n, inner dimension k
  int mr, nw;            // word rows ceil(m / dq1), word columns ceil(n / dt1)
  uint32_t dq1, dt1, s;  // rows per A word, columns per B word, Theta = Q^s
  uint32_t b, ndig;      // Q = 2^b, digits per product word
  int piece_steps;       // k-steps of 4 per piece (split form only)
  uint32_t w;            // field width of R (split form only)
  int refold;            // pieces added into R between re-reductions (split form only)
};

// Packed rows of A for full compression: CA[r][l] = sum_{i < dq1} A[r dq1 + i][l] Q^i (rows past
// m taken as zero), consecutive threads on consecutive l.  Residues >= p set ERR_RANGE.
__global__ void k_pack_rows(const uint8_t* __restrict__ A, int lda, double* __restrict__ CA, int m, int k, int mr,
                            uint32_t dq1, uint32_t b, uint32_t p, uint32_t* err) {
  const uint64_t total = (uint64_t)mr * k;
  uint32_t bad = 0;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / k), l = (int)(idx % k);
    uint64_t w = 0;
    for (int i = (int)dq1 - 1; i >= 0; --i) {
      const int row = r * (int)dq1 + i;
      const uint32_t v = row < m ? A[(size_t)row * lda + l] : 0u;
      bad |= v >= p;
      w = (w << b) | v;
    }
    CA[idx] = __ull2double_rn(w);     // exact: below 2^52
  }
  if (bad) flag_error(err, ERR_RANGE);
}

template <int TM, int TN, bool SPLIT>
__global__ void __launch_bounds__(128) k_mm_fullsplit(const uint8_t* __restrict__ A, int lda,
                                                      const double* __restrict__ CA, const double* __restrict__ CB,
                                                      uint8_t* __restrict__ C, int ldc, FsParams F,
                                                      RedqParams P, RedqParams Pw, uint32_t* err) {
  __shared__ uint8_t ptab[1024];
  __shared__ uint8_t ptab_w[1024];
  fill_pair_table(ptab, P);
  fill_pair_table(ptab_w, Pw);
  __syncthreads();
  Corrector corr, corr_w;
  corr.init(P, ptab);
  corr_w.init(Pw, ptab_w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.y * 2 + (warp >> 1)) * (8 * TM);   // first word row of this warp
  const int c0 = (blockIdx.x * 2 + (warp & 1)) * (8 * TN);    // first word column
  const uint32_t p = P.p;
  double acc[TM][TN][2];
  uint64_t R[SPLIT ? TM : 1][SPLIT ? TN : 1][2];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[i][j][0] = acc[i][j][1] = 0.0;
      if (SPLIT) R[SPLIT ? i : 0][SPLIT ? j : 0][0] = R[SPLIT ? i : 0][SPLIT ? j : 0][1] = 0;
    }
  const uint64_t qmask = (1ull << F.b) - 1ull;

  // the accumulator's digits moved into R's wider fields (split form)
  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t x = (uint64_t)acc[i][j][h];   // exact integer below 2^52
          uint64_t add = 0;
          for (uint32_t d = 0; d < F.ndig; ++d) add += ((x >> (d * F.b)) & qmask) << (d * F.w);
          if (SPLIT) R[SPLIT ? i : 0][SPLIT ? j : 0][h] += add;
          acc[i][j][h] = 0.0;
        }
  };
  // every field of R replaced by its residue (REDQ at q = 2^w); all lanes take part
  auto rereduce = [&]() {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint64_t& x = R[SPLIT ? i : 0][SPLIT ? j : 0][h];
          uint64_t y = 0;
          redq_word<uint64_t>(x, Pw, corr_w, [&](uint32_t d, uint32_t mu) { y |= (uint64_t)mu << (d * F.w); });
          x = y;
        }
  };

  uint32_t bad = 0;
  int in_piece = 0, folds = 0;
  for (int k0 = 0; k0 < F.k; k0 += 4) {
    const int kk = k0 + t;
    const bool kin = kk < F.k;
    double a[TM], bw[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int wr = r0 + 8 * i + g;
      if (CA) {                                          // packed rows (full compression)
        a[i] = (kin && wr < F.mr) ? CA[(size_t)wr * F.k + kk] : 0.0;
      } else {                                           // one row per word (right compression)
        const uint32_t v = (kin && wr < F.m) ? A[(size_t)wr * lda + kk] : 0u;
        bad |= v >= p;
        a[i] = (double)v;
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int wc = c0 + 8 * j + g;
      bw[j] = (kin && wc < F.nw) ? CB[(size_t)kk * F.nw + wc] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                     : "d"(a[i]), "d"(bw[j]));
    if (SPLIT && ++in_piece == F.piece_steps) {
      in_piece = 0;
      fold();
      if (++folds == F.refold) {
        folds = 0;
        rereduce();
      }
    }
  }
  if (SPLIT && in_piece) fold();
  if (bad) flag_error(err, ERR_RANGE);

  // epilogue: the CTA's words staged in shared memory, then REDQ of every word in a rolled loop
  // (all lanes of each warp take part in every lookup); digit d of word (wr, wc) is
  // C[wr dq1 + d mod s][wc dt1 + d div s] when d mod s < dq1
  constexpr int CM = 16 * TM, CN = 16 * TN;
  __shared__ uint64_t sw[CM * CN];
  const int lr0 = (warp >> 1) * (8 * TM), lc0 = (warp & 1) * (8 * TN);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        sw[(lr0 + 8 * i + g) * CN + lc0 + 8 * j + 2 * t + h] =
            SPLIT ? R[SPLIT ? i : 0][SPLIT ? j : 0][h] : (uint64_t)__double_as_longlong(acc[i][j][h]);
  __syncthreads();
  const int WR0 = blockIdx.y * CM, WC0 = blockIdx.x * CN;
#pragma unroll 1
  for (int idx = threadIdx.x; idx < CM * CN; idx += blockDim.x) {
    const int wr = WR0 + idx / CN, wc = WC0 + idx % CN;
    const bool own = wr < F.mr && wc < F.nw;
    auto emit = [&](uint32_t d, uint32_t mu) {
      const uint32_t i = d % F.s, j = d / F.s;
      const int row = wr * (int)F.dq1 + (int)i, col = wc * (int)F.dt1 + (int)j;
      if (own && i < F.dq1 && row < F.m && col < F.n) C[(size_t)row * ldc + col] = (uint8_t)mu;
    };
    if (SPLIT) redq_word<uint64_t>(sw[idx], Pw, corr_w, emit);
    else redq_word<double>(__longlong_as_double((long long)sw[idx]), P, corr, emit);
  }
}

// ------------------------------------------------------------------ planner

// Largest value of a word whose ndig digits are all at most D, at q = 2^b, below 2^52?
static bool digits_fit(uint64_t D, uint32_t b, uint32_t ndig) {
  if ((uint64_t)b * ndig > 120) return false;
  unsigned __int128 tot = 0;
  for (uint32_t d = 0; d < ndig; ++d) tot += (unsigned __int128)D << (d * b);
  return tot < ((unsigned __int128)1 << 52);
}

static uint32_t q_bits(uint64_t D) {   // smallest b with 2^b > D (Eq. lower, strict)
  uint32_t b = 1;
  while (b < 63 && (1ull << b) <= D) ++b;
  return b;
}

// The longest piece (a multiple of 4, at most 2^30) for which ndig digits of at most
// L (p-1)^2 fit below 2^52 at q = 2^b(L), or 0.  `need_fold`: R's fields must be wider than b.
static uint64_t longest_piece(uint32_t p, uint32_t ndig, bool need_fold) {
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  uint64_t lo = 0, hi = 1ull << 30;   // the predicate is monotone in L
  auto ok = [&](uint64_t L) {
    const uint64_t D = L * pp;
    const uint32_t b = q_bits(D);
    if (!digits_fit(D, b, ndig)) return false;
    return !need_fold || 64 / ndig > b;
  };
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (ok(mid)) lo = mid;
    else hi = mid - 1;
  }
  return lo & ~3ull;
}

// Pieces of balanced length (a multiple of 4) no longer than Lmax covering k.
static uint64_t balanced_piece(uint64_t k, uint64_t Lmax) {
  const uint64_t np = (k + Lmax - 1) / Lmax;
  return ((k + np - 1) / np + 3) & ~3ull;
}

static constexpr uint64_t MIN_PIECE = 256;   // pieces shorter than this cost more folds than they save

fp_status split_choose(uint32_t p, uint64_t k, uint32_t* b, uint32_t* e, uint32_t* piece) {
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  for (uint32_t ee = 12; ee >= 1; --ee) {
    if (digits_fit(k * pp, q_bits(k * pp), ee)) {
      *e = ee;                                  // no split needed
      *b = q_bits(k * pp);
      *piece = (uint32_t)std::min<uint64_t>(k, 0xffffffffu);
      return FP_OK;
    }
    const uint64_t Lmax = longest_piece(p, ee, true);
    if (Lmax >= std::min<uint64_t>(k, MIN_PIECE) && Lmax >= 4) {
      const uint64_t L = balanced_piece(k, Lmax);
      *e = ee;
      *b = q_bits(L * pp);
      *piece = (uint32_t)L;
      return FP_OK;
    }
  }
  set_error("SPLIT_F64: no packing fits (k=%llu p=%u)", (unsigned long long)k, p);
  return FP_EBOUND;
}

fp_status full_choose(uint32_t p, uint64_t k, uint32_t* b, uint32_t* dq1, uint32_t* dt1, uint32_t* piece) {
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  // (dq1, dt1) with dq1 <= dt1, both >= 2, the most digits first, then the most balanced; pieces
  // of at least min(k, 256) entries, else (larger p) of at least 16
  for (const uint64_t min_piece : {MIN_PIECE, (uint64_t)16})
  for (uint32_t prod = 16; prod >= 4; --prod) {
    for (uint32_t q1 = 8; q1 >= 2; --q1) {
      if (prod % q1 || prod / q1 < q1) continue;
      const uint32_t t1 = prod / q1, nd = q1 * t1;
      if (digits_fit(k * pp, q_bits(k * pp), nd)) {
        *dq1 = q1;
        *dt1 = t1;
        *b = q_bits(k * pp);
        *piece = (uint32_t)std::min<uint64_t>(k, 0xffffffffu);
        return FP_OK;
      }
      const uint64_t Lmax = longest_piece(p, nd, true);
      if (Lmax >= std::min<uint64_t>(k, min_piece) && Lmax >= 4) {
        const uint64_t L = balanced_piece(k, Lmax);
        *dq1 = q1;
        *dt1 = t1;
        *b = q_bits(L * pp);
        *piece = (uint32_t)L;
        return FP_OK;
      }
    }
  }
  set_error("FULL_F64 needs two rows and two columns per word: k (p-1)^2 too large (k=%llu p=%u)",
            (unsigned long long)k, p);
  return FP_EBOUND;
}

// ------------------------------------------------------------------ launcher

static fp_status launch_fs(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                           const uint8_t* B, int ldb, uint8_t* C, int ldc, uint32_t b, uint32_t dq1, uint32_t dt1,
                           uint32_t piece, cudaStream_t st) {
  FsParams F{};
  F.m = m;
  F.n = n;
  F.k = k;
  F.dq1 = dq1;
  F.dt1 = dt1;
  F.s = dq1;
  F.b = b;
  F.ndig = F.s * (dt1 - 1) + dq1;
  F.mr = (m + (int)dq1 - 1) / (int)dq1;
  F.nw = (n + (int)dt1 - 1) / (int)dt1;
  const bool split = (uint64_t)piece < (uint64_t)k;
  // packed operands in context scratch: B's words (dt1 columns at Theta = 2^(s b)) always, A's
  // words (dq1 rows at Q) for full compression
  const size_t cb_bytes = ((size_t)k * F.nw * sizeof(double) + 255) & ~(size_t)255;
  const size_t ca_bytes = dq1 > 1 ? (size_t)F.mr * k * sizeof(double) : 0;
  fp_status st_s = ensure_scratch(ctx, cb_bytes + ca_bytes, 0, st);
  if (st_s != FP_OK) return st_s;
  double* CB = (double*)ctx->scratch;
  double* CA = dq1 > 1 ? (double*)((uint8_t*)ctx->scratch + cb_bytes) : nullptr;
  st_s = launch_pack_cb(ctx, p, k, n, B, ldb, b * F.s, dt1, FP_WORD_F64, CB, st);
  if (st_s != FP_OK) return st_s;
  if (CA) {
    const uint64_t total = (uint64_t)F.mr * k;
    const int pg = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->num_sms * 16);
    FP_LAUNCH(ctx, "k_pack_rows", st, k_pack_rows<<<pg, 256, 0, st>>>(A, lda, CA, m, k, F.mr, dq1, b, p, ctx->d_err));
    FP_CUDA(cudaGetLastError());
  }
  RedqParams P = make_redq(p, b, F.ndig);
  RedqParams Pw = P;
  if (split) {
    F.piece_steps = (int)(piece / 4);
    F.w = std::min<uint32_t>(64 / F.ndig, 63);
    // fields start below p after a re-reduction and grow by at most 2^b - 1 per piece
    const uint64_t room = ((1ull << F.w) - 1) - (p - 1);
    F.refold = (int)std::min<uint64_t>(room / ((1ull << b) - 1), 1u << 20);
    FP_CHECK(F.refold >= 1 && piece % 4 == 0, FP_EBOUND, "split planner: no room for a piece (b=%u w=%u)", b, F.w);
    Pw = make_redq(p, F.w, F.ndig);
  }
  const uint64_t warps_big = (uint64_t)((F.mr + 31) / 32) * ((F.nw + 31) / 32);
  const bool big = warps_big >= (uint64_t)ctx->num_sms * 8;
  const int T = big ? 4 : 2;
  dim3 grid((F.nw + 16 * T - 1) / (16 * T), (F.mr + 16 * T - 1) / (16 * T));
  FP_CHECK(grid.y <= 65535u, FP_EINVAL, "matrix too tall for the FP64 word grid");
  const char* nm = split ? "k_mm_fullsplit_split" : "k_mm_fullsplit";
  if (big) {
    if (split) FP_LAUNCH(ctx, nm, st, k_mm_fullsplit<4, 4, true><<<grid, 128, 0, st>>>(A, lda, CA, CB, C, ldc, F, P, Pw, ctx->d_err));
    else FP_LAUNCH(ctx, nm, st, k_mm_fullsplit<4, 4, false><<<grid, 128, 0, st>>>(A, lda, CA, CB, C, ldc, F, P, Pw, ctx->d_err));
  } else {
    if (split) FP_LAUNCH(ctx, nm, st, k_mm_fullsplit<2, 2, true><<<grid, 128, 0, st>>>(A, lda, CA, CB, C, ldc, F, P, Pw, ctx->d_err));
    else FP_LAUNCH(ctx, nm, st, k_mm_fullsplit<2, 2, false><<<grid, 128, 0, st>>>(A, lda, CA, CB, C, ldc, F, P, Pw, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

fp_status mm_full(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                  int ldb, uint8_t* C, int ldc, cudaStream_t st) {
  uint32_t b, dq1, dt1, piece;
  fp_status s = full_choose(p, (uint64_t)k, &b, &dq1, &dt1, &piece);
  if (s != FP_OK) return s;
  return launch_fs(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, b, dq1, dt1, piece, st);
}

fp_status mm_split(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                   int ldb, uint8_t* C, int ldc, cudaStream_t st) {
  uint32_t b, e, piece;
  fp_status s = split_choose(p, (uint64_t)k, &b, &e, &piece);
  if (s != FP_OK) return s;
  return launch_fs(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, b, 1, e, piece, st);
}

}  // namespace fpd

extern "C" fp_status fp_mm_full_choose(uint32_t p, uint64_t kdim, uint32_t* b, uint32_t* dq1, uint32_t* dt1,
                                       uint32_t* piece) {
  FP_CHECK(b && dq1 && dt1 && piece, FP_EINVAL, "fp_mm_full_choose: null output");
  FP_CHECK(p >= 2 && p <= 251 && fpd::is_prime(p), FP_EINVAL, "fp_mm_full_choose: p=%u not a prime <= 251", p);
  FP_CHECK(kdim >= 1 && kdim <= (1ull << 30), FP_EINVAL, "fp_mm_full_choose: kdim outside [1, 2^30]");
  return fpd::full_choose(p, kdim, b, dq1, dt1, piece);
}
