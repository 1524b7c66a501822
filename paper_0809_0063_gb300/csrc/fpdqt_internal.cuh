// Internal declarations shared by the CUDA translation units of libfpdqt.
//
// Device side: the REDQ routine (Algorithm 2) with the FDIV division (Algorithm FDIV,
// case 3 of Table "fdiv": inverse rounded up, product rounded down, exact below 2^(beta-1))
// and the tabulated correction (Sec. 3.4-3.5), for FP64, FP32, u64 and u32 words.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/fpdqt.h"

#define FP_NUM_SMS_HINT 152

// ------------------------------------------------------------------ host error plumbing
namespace fpd {

void set_error(const char* fmt, ...);
fp_status cuda_fail(cudaError_t e, const char* what);

#define FP_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fpd::cuda_fail(e_, #call);   \
  } while (0)

#define FP_CHECK(cond, status, ...)          \
  do {                                       \
    if (!(cond)) {                           \
      fpd::set_error(__VA_ARGS__);           \
      return (status);                       \
    }                                        \
  } while (0)

// Device-side sticky error bits (ORed into ctx->d_err).
enum : uint32_t { ERR_RANGE = 1u, ERR_TIMEOUT = 2u };

bool is_prime(uint32_t p);

// Invariant integer division by p (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994, Sec. 4): for p not a power of two, with l = ceil(log2 p),
// m = floor(2^N (2^l - p) / p) + 1, floor(n/p) = (t + ((n - t) >> 1)) >> (l - 1) where
// t = mulhi(m, n).  For p a power of two it is a shift by sh.
struct DivP {
  uint64_t m64;   // multiplier for 64-bit dividends
  uint32_t m32;   // multiplier for 32-bit dividends
  uint32_t l;     // ceil(log2 p)
  uint32_t pow2;  // 1 if p is a power of two
  uint32_t sh;    // log2 p when pow2
};
DivP make_divp(uint32_t p);

// Word helpers.
int word_beta(uint32_t word);      // exact integer range in bits (52, 64, 23, 32)
size_t word_bytes(uint32_t word);

}  // namespace fpd

// ------------------------------------------------------------------ context
struct fp_ctx_s {
  int device = 0;
  int num_sms = FP_NUM_SMS_HINT;
  uint32_t* d_err = nullptr;        // sticky device error flag
  void* scratch = nullptr;          // packed operands, partials
  size_t scratch_bytes = 0;
  void* scratch2 = nullptr;
  size_t scratch2_bytes = 0;
  // set once a call has run inside a stream capture: from then on scratch that grows is not
  // freed (a captured graph may still refer to it) but kept here until the context is destroyed
  bool captured = false;
  std::vector<void*> retired;
  std::mutex mu;
  // autotuner cache: key -> chosen variant
  std::unordered_map<uint64_t, int> tune;
  int autotune = 1;
  // instrumentation: launch count and optional per-launch event pairs
  uint64_t launches = 0;
  int prof = 0;
  struct Rec { const char* name; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::mutex pmu;
  // pinned host staging for per-call uploads (batch plans, job lists), one buffer per use slot:
  // a slot is rewritten only after the copy that last read it has run (its event), so an upload
  // never waits for the kernels before it in the stream (a pageable copy would)
  static constexpr int PIN_SLOTS = 4;
  void* pin[PIN_SLOTS] = {};
  size_t pin_bytes[PIN_SLOTS] = {};
  cudaEvent_t pin_ev[PIN_SLOTS] = {};
};

namespace fpd {
// Context scratch slot `which` grown to at least `bytes`.  Inside a stream capture on `st` a
// growth is refused (FP_EUNSUPPORTED: it would free memory and synchronise); a call made once
// outside the capture sizes it.
fp_status ensure_scratch(fp_ctx ctx, size_t bytes, int which, cudaStream_t st);
bool stream_capturing(cudaStream_t st);
// Asynchronous host-to-device copy of `bytes` from `src` through the context's pinned staging
// slot `slot` (0 .. PIN_SLOTS-1); `src` may be reused as soon as the call returns.
fp_status upload_staged(fp_ctx ctx, int slot, void* dst, const void* src, size_t bytes, cudaStream_t st);
void launch_begin(fp_ctx ctx, const char* name, cudaStream_t st);
void launch_end(fp_ctx ctx, cudaStream_t st);
// Launch a kernel through the context's instrumentation (launch count, optional events).
#define FP_LAUNCH(ctx, name, st, ...)      \
  do {                                     \
    fpd::launch_begin((ctx), (name), (st)); \
    __VA_ARGS__;                           \
    fpd::launch_end((ctx), (st));          \
  } while (0)
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
}  // namespace fpd

// ------------------------------------------------------------------ device REDQ
namespace fpd {

// Parameters of one REDQ instance, passed by value to kernels.
struct RedqParams {
  uint32_t p;       // prime
  uint32_t b;       // q = 2^b
  uint32_t ndig;    // residues recovered per word
  uint32_t c;       // (-q) mod p: superdiagonal of the correction matrix Q_k (Sec. 3.4)
  uint32_t mode;    // correction: 0 none (p | q), 1 shuffle Q_2 table (p^3 <= 32),
                    // 2 shuffle pair table (p^2 <= 32), 3 shared-memory pair table, 4 arithmetic
  uint32_t pad;
  double invp_d;    // RU(1/p) in binary64
  float invp_f;     // RU(1/p) in binary32
  DivP dv;
};

RedqParams make_redq(uint32_t p, uint32_t b, uint32_t ndig);

enum : uint32_t { CORR_NONE = 0, CORR_SHFL3 = 1, CORR_SHFL2 = 2, CORR_SMEM2 = 3, CORR_ARITH = 4 };

// floor(n / p) for the invariant p.
__device__ __forceinline__ uint32_t divp32(uint32_t n, const DivP& d) {
  if (d.pow2) return n >> d.sh;
  uint32_t t = __umulhi(d.m32, n);
  return (t + ((n - t) >> 1)) >> (d.l - 1);
}
__device__ __forceinline__ uint64_t divp64(uint64_t n, const DivP& d) {
  if (d.pow2) return n >> d.sh;
  uint64_t t = __umul64hi(d.m64, n);
  return (t + ((n - t) >> 1)) >> (d.l - 1);
}
__device__ __forceinline__ uint32_t modp32(uint32_t n, const DivP& d, uint32_t p) {
  return n - p * divp32(n, d);
}

// REDQ COMPRESSION quotient s = floor(r / p) (Algorithm 2, first line) per word type.
// FP words use Algorithm FDIV in case 3 of Table "fdiv": x = RD(r * RU(1/p)), floor(x);
// exact for r < 2^(beta-1), which the planner guarantees for every packed word.
template <typename W> struct WordOps;

template <> struct WordOps<double> {
  __device__ __forceinline__ static uint64_t to_u64(double r) { return (uint64_t)r; }
  __device__ __forceinline__ static uint64_t quot(double r, const RedqParams& P) {
    return (uint64_t)__dmul_rd(r, P.invp_d);
  }
  __device__ __forceinline__ static double from_u64(uint64_t v) { return __ull2double_rn(v); }
};
template <> struct WordOps<float> {
  __device__ __forceinline__ static uint64_t to_u64(float r) { return (uint64_t)__float2uint_rz(r); }
  __device__ __forceinline__ static uint64_t quot(float r, const RedqParams& P) {
    return (uint64_t)__float2uint_rz(__fmul_rd(r, P.invp_f));
  }
  __device__ __forceinline__ static float from_u64(uint64_t v) { return __uint2float_rn((uint32_t)v); }
};
template <> struct WordOps<uint64_t> {
  __device__ __forceinline__ static uint64_t to_u64(uint64_t r) { return r; }
  __device__ __forceinline__ static uint64_t quot(uint64_t r, const RedqParams& P) { return divp64(r, P.dv); }
  __device__ __forceinline__ static uint64_t from_u64(uint64_t v) { return v; }
};
template <> struct WordOps<uint32_t> {
  __device__ __forceinline__ static uint64_t to_u64(uint32_t r) { return r; }
  __device__ __forceinline__ static uint64_t quot(uint32_t r, const RedqParams& P) {
    return divp32(r, P.dv);
  }
  __device__ __forceinline__ static uint32_t from_u64(uint64_t v) { return (uint32_t)v; }
};

// Per-thread state of the correction lookup.  Built once per kernel (the shuffle tables
// hold one entry per lane; the shared table is filled by the caller's block).
struct Corrector {
  uint32_t lane_val;           // shuffle-table entry held by this lane
  const uint8_t* smem;         // pair table in shared memory (mode CORR_SMEM2)

  __device__ __forceinline__ void init(const RedqParams& P, const uint8_t* sm) {
    smem = sm;
    lane_val = 0;
    uint32_t lane = threadIdx.x & 31u;
    uint32_t p = P.p;
    if (P.mode == CORR_SHFL3 && lane < p * p * p) {
      // Example tmto: the 2x3 map underline{Q}_2 on (u0,u1,u2) -> (u0-q u1, u1-q u2) mod p,
      // indexed by u0 + u1 p + u2 p^2 (Note on Indexing).
      uint32_t u0 = lane % p, u1 = (lane / p) % p, u2 = lane / (p * p);
      uint32_t a = (u0 + P.c * u1) % p, b2 = (u1 + P.c * u2) % p;
      lane_val = a | (b2 << 8);
    } else if (P.mode == CORR_SHFL2 && lane < p * p) {
      uint32_t u0 = lane % p, u1 = lane / p;
      lane_val = (u0 + P.c * u1) % p;
    }
  }
  // mu_i = (u_i - q u_{i+1}) mod p for one pair.
  __device__ __forceinline__ uint32_t pair(uint32_t ui, uint32_t un, const RedqParams& P) const {
    switch (P.mode) {
      case CORR_SHFL2: return __shfl_sync(0xffffffffu, lane_val, ui + P.p * un);
      case CORR_SMEM2: return smem[ui + P.p * un];
      case CORR_ARITH: return modp32(ui + P.c * un, P.dv, P.p);
      default: return ui;
    }
  }
};

// i-th REDQ compression residue u_i = floor(r/q^i) - p floor(s/q^i) (Algorithm 2).  Since
// 0 <= u_i < p <= q (Theorem REDQ), only the low b bits of the difference are needed, so the
// subtraction is done modulo 2^32 and masked.
__device__ __forceinline__ uint32_t redq_u(uint64_t r, uint64_t s, uint32_t i, const RedqParams& P) {
  uint32_t sh = i * P.b;
  uint32_t rr = sh < 64 ? (uint32_t)(r >> sh) : 0u;
  uint32_t ss = sh < 64 ? (uint32_t)(s >> sh) : 0u;
  return (rr - P.p * ss) & ((P.b >= 32) ? 0xffffffffu : ((1u << P.b) - 1u));
}

// u_i for words below 2^32 (FP32 / u32 words): one 32-bit shift pair per residue.
__device__ __forceinline__ uint32_t redq_u32(uint32_t r, uint32_t s, uint32_t i, const RedqParams& P) {
  const uint32_t sh = i * P.b;
  const uint32_t rr = sh < 32 ? (r >> sh) : 0u;
  const uint32_t ss = sh < 32 ? (s >> sh) : 0u;
  return (rr - P.p * ss) & ((P.b >= 32) ? 0xffffffffu : ((1u << P.b) - 1u));
}

// Full REDQ_ndig of one word: calls emit(i, mu_i) for i = 0..ndig-1 in increasing order.
// All 32 lanes of the warp must call this together (shuffle tables); ndig, mode uniform.
template <typename W, typename Emit>
__device__ __forceinline__ void redq_word(W rw, const RedqParams& P, const Corrector& C, Emit emit) {
  const uint64_t r64 = WordOps<W>::to_u64(rw);
  const uint64_t s64 = WordOps<W>::quot(rw, P);
  constexpr bool narrow = sizeof(W) == 4;      // word and quotient fit 32 bits
  auto U = [&](uint32_t i) -> uint32_t {
    return narrow ? redq_u32((uint32_t)r64, (uint32_t)s64, i, P) : redq_u(r64, s64, i, P);
  };
  const uint32_t nd = P.ndig;
  if (P.mode == CORR_NONE) {
    for (uint32_t i = 0; i < nd; ++i) emit(i, U(i));
    return;
  }
  if (P.mode == CORR_SHFL3) {
    // two residues per lookup (Example tmto with j = 3)
    uint32_t u0 = U(0);
    uint32_t i = 0;
    for (; i + 1 < nd; i += 2) {
      uint32_t u1 = U(i + 1);
      uint32_t u2 = (i + 2 < nd) ? U(i + 2) : 0u;
      uint32_t v = __shfl_sync(0xffffffffu, C.lane_val, u0 + P.p * u1 + P.p * P.p * u2);
      emit(i, v & 0xffu);
      if (i + 2 < nd) {
        emit(i + 1, v >> 8);
      } else {
        emit(i + 1, u1);       // top residue: mu_d = u_d
      }
      u0 = u2;
    }
    if (i < nd) emit(i, u0);   // nd odd: the last one is the top residue
    return;
  }
  uint32_t u = U(0);
  for (uint32_t i = 0; i < nd; ++i) {
    if (i + 1 < nd) {
      uint32_t un = U(i + 1);
      emit(i, C.pair(u, un, P));
      u = un;
    } else {
      emit(i, u);
    }
  }
}

// REDQ_2 of a 32-bit word (two residues), unrolled for epilogues that pack results into
// registers.  Same steps as redq_word; all lanes of the warp must call it together.
__device__ __forceinline__ void redq2_u32(uint32_t w, const RedqParams& P, const Corrector& C, uint32_t& mu0,
                                          uint32_t& mu1) {
  const uint32_t s = divp32(w, P.dv);
  const uint32_t mask = (P.b >= 32) ? 0xffffffffu : ((1u << P.b) - 1u);
  const uint32_t u0 = (w - P.p * s) & mask;
  const uint32_t u1 = ((w >> P.b) - P.p * (s >> P.b)) & mask;
  mu1 = u1;
  if (P.mode == CORR_NONE) mu0 = u0;
  else if (P.mode == CORR_SHFL3) mu0 = __shfl_sync(0xffffffffu, C.lane_val, u0 + P.p * u1) & 0xffu;
  else mu0 = C.pair(u0, u1, P);
}

// Fill the shared pair table (mode CORR_SMEM2) cooperatively: T[u0 + p u1] = (u0 + c u1) mod p.
__device__ __forceinline__ void fill_pair_table(uint8_t* T, const RedqParams& P) {
  if (P.mode != CORR_SMEM2) return;
  for (uint32_t idx = threadIdx.x; idx < P.p * P.p; idx += blockDim.x) {
    uint32_t u0 = idx % P.p, u1 = idx / P.p;
    T[idx] = (uint8_t)((u0 + P.c * u1) % P.p);
  }
}

// Packs src[0..k) in blocks of d+1 coefficients: word i = sum_j src[i(d+1) + j] q^j for
// i < nwords (zero past k), written to w[i]; residues >= p set bad.
__device__ __forceinline__ void fqt_pack(const uint8_t* __restrict__ src, uint32_t k, uint32_t d1, uint32_t nwords,
                                         const RedqParams& P, uint64_t* w, uint32_t& bad) {
  for (uint32_t i = threadIdx.x; i < nwords; i += blockDim.x) {
    uint64_t v64 = 0;
    for (int j = (int)d1 - 1; j >= 0; --j) {
      uint32_t idx = i * d1 + j;
      uint32_t v = idx < k ? src[idx] : 0u;
      bad |= v >= P.p;
      v64 = (v64 << P.b) | v;
    }
    w[i] = v64;
  }
}

// REDQ_{2d+1} of the nw product words word_at(o) into res, then the overlap of consecutive
// blocks: coefficient j = res[j / (d+1)][j mod (d+1)] + res[j / (d+1) - 1][j mod (d+1) + d + 1]
// mod p, for j < kc.  All threads of the block call it (whole warps run the REDQ loop, so the
// shuffle-table lookups see 32 active lanes).
template <typename WordAt>
__device__ __forceinline__ void fqt_reduce_product(WordAt word_at, uint32_t nw, uint32_t kc, uint32_t d1,
                                                   const RedqParams& P, const Corrector& C, uint8_t* res,
                                                   uint8_t* __restrict__ Cout) {
  const uint32_t nd = 2 * d1 - 1;               // residues per output word
  for (uint32_t base = 0; base < nw; base += blockDim.x) {
    uint32_t o = base + threadIdx.x;
    const bool own = o < nw;
    uint64_t acc = own ? word_at(o) : 0;
    uint8_t* out = res + (own ? o : 0) * nd;
    redq_word<uint64_t>(acc, P, C, [&](uint32_t i, uint32_t mu) { if (own) out[i] = (uint8_t)mu; });
  }
  __syncthreads();
  // j / d1 = umulhi(j, ceil(2^32 / d1)), exact for j d1 < 2^32 (the multiplier needs d1 > 1)
  const uint32_t md = d1 > 1 ? 0xffffffffu / d1 + 1u : 0u;
  for (uint32_t j = threadIdx.x; j < kc; j += blockDim.x) {
    uint32_t o = d1 > 1 ? __umulhi(j, md) : j, r = j - o * d1;
    uint32_t v = o < nw ? res[o * nd + r] : 0u;
    if (o >= 1 && r + d1 < nd) v += res[(o - 1) * nd + r + d1];
    if (v >= P.p) v -= P.p;
    Cout[j] = (uint8_t)v;
  }
}

// Blocked FQT (Sec. 5.2): P = sum_i P_i (X^{d+1})^i with each P_i (d+1 coefficients) in one
// u64 word at q = 2^b; output word t = sum_i P_i Q_{t-i} accumulated in the word (delayed
// reduction, the planner keeps every digit below q), then REDQ_{2d+1}; the residues of words t
// and t-1 overlap on d coefficients and are added mod p.  One block per product; the shared
// buffers wa, wb (1024 words each), res (4160 bytes) and the correction table are the
// caller's.  All threads of the block must call it.
__device__ __forceinline__ void fqt_block_product(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                  uint8_t* __restrict__ Cout, uint32_t ka, uint32_t kb, uint32_t d1,
                                  const RedqParams& P, const Corrector& C, uint64_t* wa, uint64_t* wb,
                                  uint8_t* res, uint32_t& bad) {
  const uint32_t na = (ka + d1 - 1) / d1, nb = (kb + d1 - 1) / d1;
  __syncthreads();
  fqt_pack(A, ka, d1, na, P, wa, bad);
  fqt_pack(B, kb, d1, nb, P, wb, bad);
  __syncthreads();
  fqt_reduce_product(
      [&](uint32_t o) {
        uint32_t lo = o + 1 > nb ? o + 1 - nb : 0;
        uint32_t hi = o < na - 1 ? o : na - 1;
        uint64_t acc = 0;
        for (uint32_t i = lo; i <= hi; ++i) acc += wa[i] * wb[o - i];
        return acc;
      },
      na + nb - 1, ka + kb - 1, d1, P, C, res, Cout);
}

// Sticky error reporting from device code.
__device__ __forceinline__ void flag_error(uint32_t* err, uint32_t bits) {
  if (err) atomicOr(err, bits);
}

}  // namespace fpd

// ------------------------------------------------------------------ uneven-batch plan records
namespace fpd {
// One instance of the persistent uneven-batch kernel (dense row-major operands).
struct BInst {
  const uint8_t* A;
  const uint8_t* B;
  uint8_t* C;
  uint32_t kind;     // 0 matmul, 1 dot
  uint32_t p, m, n, k;
  uint32_t packed;   // 1: two residues per fp16 operand word
  uint32_t nw;       // output words per row (n or ceil(n/2))
  uint32_t plain_chunk_steps;  // k-steps per fold for the plain path
  RedqParams P;      // REDQ_2 at q = 2^16 (packed) / mod p (plain)
};

struct BItem {
  uint32_t inst;
  uint16_t tm, tn;
};

}  // namespace fpd

// ------------------------------------------------------------------ launchers (per .cu)
namespace fpd {
bool fqt_params(uint32_t p, uint32_t ka, uint32_t kb, uint32_t* d1, uint32_t* b);
fp_status launch_pack(fp_ctx ctx, const fp_dqt_params& prm, const uint8_t* coeffs, void* words,
                      size_t count, cudaStream_t st);
fp_status launch_unpack(fp_ctx ctx, const fp_dqt_params& prm, const void* words, uint8_t* coeffs,
                        size_t count, cudaStream_t st);
fp_status launch_polymul(fp_ctx ctx, uint32_t p, const uint8_t* A, uint32_t da, const uint8_t* B,
                         uint32_t db, uint8_t* C, size_t batch, int algo, cudaStream_t st);
fp_status launch_matmul(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                        const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, cudaStream_t st);
fp_status launch_pack_cb(fp_ctx ctx, uint32_t p, int k, int n, const uint8_t* B, int ldb, uint32_t b,
                         uint32_t e, uint32_t word, void* CB, cudaStream_t st);
fp_status launch_dot(fp_ctx ctx, uint32_t p, const uint8_t* u, const uint8_t* v, size_t n,
                     uint32_t* out, int algo, cudaStream_t st);
fp_status mm_bound_check(uint32_t p, int k, int algo);
// full compression (Sec. 7.5) and right compression with a split inner dimension (Sec. 7.6) on
// FP64 words (k_full.cu): planners and the products
fp_status full_choose(uint32_t p, uint64_t k, uint32_t* b, uint32_t* dq1, uint32_t* dt1, uint32_t* piece);
fp_status split_choose(uint32_t p, uint64_t k, uint32_t* b, uint32_t* e, uint32_t* piece);
fp_status mm_full(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                  int ldb, uint8_t* C, int ldc, cudaStream_t st);
fp_status mm_split(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                   int ldb, uint8_t* C, int ldc, cudaStream_t st);
// grouped e4m3 tensor-core product (k_tcg.cu)
bool f8_direct_ok(uint32_t p, int k, const uint8_t* A, int lda, const uint8_t* B, int ldb);
fp_status launch_mm_f8_direct(fp_ctx ctx, const fp_mm_problem& x, cudaStream_t st);   // lock held
fp_status launch_mm_f8_grouped(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, cudaStream_t st);
// Plain bf16 tensor-core products of an uneven batch (k (p-1)^2 < 2^24): operands converted and
// range-checked in one launch into `scratch` (t16_batch_bytes long), then grouped launches.  Lock held.
uint64_t t16_batch_bytes(const fp_mm_problem* const* pr, size_t count);
fp_status launch_mm_t16_plain_batch(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, uint8_t* scratch,
                                    cudaStream_t st);
// Pre-tiled e4m3 products (the tensor-core share of an uneven batch).  Each operand is laid out
// by the batch's pack pass as 16 KB blocks of 128 x 128 bytes, each in the 128-byte swizzle of
// a shared-memory stage (16-byte chunk c of block row r at chunk position c ^ (r & 7)), holding
// centred residues (|c| <= p/2 <= 15) as signed e4m3 codes and zero outside the matrix:
//   A (m x k, K-major):  block (mb, kt) = rows 128 mb.., k bytes 128 kt..
//                        at At + (mb ktiles + kt) F8_BLOCK,
//   B (k x n, MN-major): block (nb, kt, h) = k rows 128 kt.., columns 256 nb + 128 h..
//                        at Bt + ((nb ktiles + kt) 2 + h) F8_BLOCK.
static constexpr int F8_BLOCK = 16384;
static constexpr int F8_PRE_CAP = 4096;     // problems per launch
struct F8PreProb {
  const uint8_t* At;
  const uint8_t* Bt;
  uint8_t* C;
  int m, n, ldc;
  int ktiles;          // ceil(k / 128)
  int klast;           // K = 32 steps holding some of the last k tile (1..4)
  int tn;              // column blocks ceil(n / 256)
  uint32_t p;
  float off18;         // p T 2^-18 with p T >= k (p/2)^2 (makes every sum non-negative), or 0
};
// prob, tile0: nprob <= F8_PRE_CAP entries in device memory, tile0 ascending from 0 (the first
// tile of each problem, tiles of a problem in row-block-major order), total tiles.  Lock held.
fp_status launch_mm_f8_pretiled(fp_ctx ctx, const F8PreProb* prob, const int* tile0, int nprob, int total,
                                cudaStream_t st);
// lock held
fp_status launch_mm_f8_grouped_locked(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, cudaStream_t st);
// grouped 16-bit tensor-core products (k_tcp.cu): packed fp16 (right compression, p <= 3)
// or plain bf16
bool f16p_ok(uint32_t p, int k);
fp_status launch_mm_t16_direct(fp_ctx ctx, const fp_mm_problem& x, bool packed, cudaStream_t st);   // lock held
fp_status launch_mm_t16_grouped(fp_ctx ctx, const fp_mm_problem* const* pr, size_t count, bool packed,
                                cudaStream_t st);
}  // namespace fpd
