/*
 * fpdqt.h -- C ABI of the packed small-prime-field library (GB300, sm_103a).
 *
 * The library computes exact products over F_p (p prime, 2 <= p <= 251) and over small
 * extension fields GF(p^k) by packing several residues into one machine word with the
 * Discrete Q-adic Transform (DQT, the map sum a_i X^i -> sum a_i q^i of Eq. dqt, Sec. 1),
 * multiplying and accumulating those words with delayed reduction (Sec. 2.2-2.3), and
 * recovering the residues with REDQ simultaneous reduction (Algorithm 2, Sec. 3) in which the
 * one division is an FP multiply by a rounded inverse (Algorithm FDIV, Table "fdiv", Sec. 4).
 * Here q = Q = 2^b (the restriction at the end of Sec. 3), except that fp_dqt_pack and
 * fp_dqt_unpack_redq also take q = p 2^b (the alternative the conclusion proposes).
 *
 * Conventions shared by every call
 *  - All array pointers are DEVICE pointers owned by the caller unless stated otherwise; the
 *    library never frees them.  Arrays are dense, row-major, uint8 per F_p residue.
 *  - Every compute call is asynchronous on the given CUDA stream (NULL = legacy default).
 *    Host-side argument checks happen before anything is enqueued; a failing check returns
 *    its status and enqueues nothing.
 *  - A context owns scratch memory that calls reuse (padded or converted operands, plans,
 *    partial sums): calls on one context are ordered by their stream, so calls issued on
 *    different streams with one context must be ordered by the caller (an event or a
 *    synchronisation between them), or use one context per stream.  The serving loop keeps
 *    its own device arena and is exempt.
 *  - Residue inputs must lie in [0, p-1].  Kernels check this on the device; a violation
 *    sets the context's sticky error flag (results are then unspecified but every memory
 *    access stays in bounds).  fp_ctx_status() synchronises the stream and reports it.
 *  - No C++ exception crosses the ABI.  fp_last_error() gives a thread-local message for
 *    the last non-FP_OK status of the calling thread.
 *  - Status codes: FP_EINVAL (bad argument), FP_EBOUND (forced parameters violate the
 *    exactness bounds of Eq. bounds / Eq. lower / Eq. upper), FP_ENOMEM, FP_ECUDA (a CUDA
 *    runtime call failed), FP_ETIMEOUT (a bounded device wait gave up), FP_EUNSUPPORTED.
 */
#ifndef FPDQT_H
#define FPDQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FP_OK = 0,
  FP_EINVAL = 1,
  FP_EBOUND = 2,
  FP_ENOMEM = 3,
  FP_ECUDA = 4,
  FP_ETIMEOUT = 5,
  FP_EUNSUPPORTED = 6
} fp_status;

/* Machine word holding a packed value.  beta = exact integer range used for the bounds:
 * F64 52 bits (FDIV case 3 of Table "fdiv" is exact below 2^(53-1)), F32 23 bits (same rule
 * with a 24-bit mantissa), U64 64 bits, U32 32 bits. */
typedef enum { FP_WORD_F64 = 0, FP_WORD_U64 = 1, FP_WORD_F32 = 2, FP_WORD_U32 = 3 } fp_word;

/* Algorithm selectors for fp_polymul_batched / fp_dot. */
enum {
  FP_ALGO_AUTO = 0,    /* planner's choice (fastest exact packed word) */
  FP_ALGO_PLAIN = 1,   /* unpacked schoolbook with delayed reduction (Eq. delayed) */
  FP_ALGO_DQT_F64 = 2, /* packed words of the given type */
  FP_ALGO_DQT_U64 = 3,
  FP_ALGO_DQT_F32 = 4,
  FP_ALGO_DQT_U32 = 5,
  FP_ALGO_KARATSUBA = 6 /* fp_polymul_batched only: the blocked FQT's u64 words multiplied as word
                           polynomials by Karatsuba splitting (Sec. 5.2, Fig. pmkara) */
};

/* Algorithm selectors for fp_matmul. */
enum {
  FP_MM_AUTO = 0,       /* fastest exact variant: PLAIN_F8 when p <= 17 and k (p-1)^2 < 2^24
                           (fastest measured on GB300 at every size); otherwise the candidate the
                           autotuner measured fastest (packed or plain) */
  FP_MM_RIGHT_F64 = 1,  /* right compression (Sec. 7.4), FP64 words, FP64 tensor cores (DMMA) */
  FP_MM_RIGHT_F32 = 2,  /* right compression, FP32 words, FFMA, inner dimension split so the
                           digit bound holds per chunk; chunks folded into an integer word */
  FP_MM_PLAIN_F64 = 3,  /* unpacked, FP64 DMMA, delayed reduction, mod p epilogue */
  FP_MM_PLAIN_F32 = 4,  /* unpacked, FFMA, delayed reduction, mod p epilogue */
  FP_MM_PLAIN_I8 = 5,   /* unpacked, u8 x u8 -> s32 tensor cores (mma.sync), mod p epilogue */
  FP_MM_PLAIN_TC = 6,   /* unpacked, tcgen05 kind::f16 (bf16 operands, fp32 accumulate) */
  FP_MM_RIGHT_TC = 7,   /* right compression on tcgen05 kind::f16: fp16 operands holding two
                           centred residues, inner dimension chunked: p <= 3 at Q = 2^10 in
                           chunks of 448 (k <= 32767); p = 5, 7 at Q = 1023 / 681 (the largest
                           Q whose pairs are exact fp16 integers; fp_mm_choose reports b = 0) in
                           chunks of 64 / 32 inner steps, any k */
  FP_MM_LEFT_F32 = 8,   /* left compression (Sec. 7.4): by transposition, (A B)^T = B^T A^T with
                           the right compression (FP32 words) of A^T, i.e. each word packs two
                           consecutive rows of A; A^T, B^T and C^T go through context scratch */
  FP_MM_PLAIN_F8 = 9,   /* unpacked, tcgen05 kind::f8f6f4, fp32 accumulate: the residue bytes
                           are read as e4m3 (r 2^-9, exact for r <= 16); p <= 17 and
                           k (p-1)^2 < 2^24.  A and B 16-byte aligned with lda, ldb multiples
                           of 16 are read in place; other layouts are first copied padded */
  FP_MM_LEFT_F64 = 10,  /* left compression by transposition with FP64 words (DMMA), e rows of A
                           per word as RIGHT_F64 packs e columns of B */
  FP_MM_CMM_F64 = 11,   /* compressed matrix multiplication by the middle product (Sec. 7.1):
                           d+1 entries of the inner dimension per FP64 word, A reversed, B
                           forward, q = 2^b > k (p-1)^2, d the largest with (2d+1) b <= 52 so
                           every word product is exact; C_ij is the digit of q^d mod p.  Needs
                           d >= 1, i.e. k (p-1)^2 < 2^17, else FP_EBOUND */
  FP_MM_FULL_F64 = 12,  /* full compression (Sec. 7.5, Eq. qtheta, Eq. dq): dq1 rows of A per FP64
                           word at Q = 2^b, dt1 columns of B per word at Theta = Q^dq1 (the
                           smallest Theta Eq. qtheta allows), DMMA product of the packed words,
                           REDQ over dq1 dt1 base-Q digits; dq1, dt1 >= 2 chosen by
                           fp_mm_full_choose, the inner dimension split into pieces (as
                           SPLIT_F64) when it is too long for a 2 x 2 packing in one piece */
  FP_MM_SPLIT_F64 = 13  /* right compression (Sec. 7.4) with the inner dimension cut into pieces
                           (Sec. 7.6, after Table comprange) that each keep the compression e of
                           a shorter product: e.g. p = 3 keeps e = 4 past k = 2047, where
                           RIGHT_F64 drops to e = 3.  Pieces' digits are added into wider fields
                           and reduced by REDQ; see fp_mm_choose for the piece length */
};

/* Forms of q in fp_dqt_params.qform. */
enum {
  FP_Q_POW2 = 0,    /* q = 2^b (Sec. 3, end: conversions by shifts, tabulated correction) */
  FP_Q_P_POW2 = 1   /* q = p 2^b (the conclusion's alternative): p divides q, so REDQ needs no
                       correction (mu_i = u_i), and floor(r / q^i) = floor(r / p^i) >> (b i)
                       makes every division one by p */
};

/* Parameters of one packed representation (Sec. 2.3): q = 2^b (or p 2^b, see qform), k residues
 * packed per operand word, ndig residues recovered per result word, n_accum products
 * accumulated.  fp_dqt_choose fills qform = FP_Q_POW2. */
typedef struct {
  uint32_t p;
  uint32_t k;
  uint32_t b;
  uint32_t ndig;
  uint32_t word;     /* fp_word */
  uint32_t qform;    /* FP_Q_POW2 or FP_Q_P_POW2 */
  uint64_t n_accum;
} fp_dqt_params;

typedef struct fp_ctx_s* fp_ctx;
typedef struct fp_gf_s* fp_gf;

/* ---------------------------------------------------------------- context and errors */

/* Create a context on CUDA device `device` (made current on the calling thread).  The
 * context owns: the sticky device error flag, scratch for packed operands (grown on demand
 * with cudaMalloc), REDQ correction tables and the plan cache.  *out receives the handle.
 * Errors: FP_EINVAL (null out / bad device), FP_ECUDA, FP_ENOMEM.
 * Resource management: no counterpart in the paper. */
fp_status fp_ctx_create(fp_ctx* out, int device);

/* Destroy a context and free everything it owns (synchronises its device first).  NULL ok.
 * Resource management: no counterpart in the paper. */
void fp_ctx_destroy(fp_ctx ctx);

/* Synchronise `stream`, then read and clear the context's sticky device error flag (no
 * counterpart in the paper: the range check of inputs that the paper assumes valid).
 * Returns FP_EINVAL if any kernel saw a residue outside [0, p-1] (or a GF index outside
 * [0, p^k)), FP_ETIMEOUT if a bounded device wait gave up, FP_ECUDA on a CUDA error. */
fp_status fp_ctx_status(fp_ctx ctx, void* stream);

/* Thread-local message describing the last error of the calling thread ("" if none); the
 * pointer stays valid until the thread's next failing call (no counterpart in the paper). */
const char* fp_last_error(void);

/* Instrumentation (no counterpart in the paper).  mode 1 starts recording a CUDA event pair
 * around every kernel the library launches on this context (on the launch stream), 0 stops,
 * 2 clears the records.  Errors: FP_EINVAL (null ctx, other modes). */
fp_status fp_ctx_profile(fp_ctx ctx, int mode);

/* Instrumentation (no counterpart in the paper): synchronises the recorded events and returns,
 * for the kernels whose name starts with `prefix` (NULL or "" = all), the number of recorded
 * launches and their summed device time in milliseconds (either output may be NULL).
 * Errors: FP_EINVAL (null ctx), FP_ECUDA. */
fp_status fp_ctx_profile_read(fp_ctx ctx, const char* prefix, uint64_t* launches, double* total_ms);

/* Instrumentation (no counterpart in the paper): the total number of kernels the library has
 * launched on this context since creation, recorded or not.  Errors: FP_EINVAL (null). */
fp_status fp_ctx_launches(fp_ctx ctx, uint64_t* count);

/* Tuning of fp_matmul's AUTO choice (no counterpart in the paper; the candidates are the
 * packings of Sec. 7 and the plain products).  When enabled (the default), the first FP_MM_AUTO call
 * for a new (p, size class) outside PLAIN_F8's rule times every exact candidate (packed tensor-core, plain
 * tensor-core, u8 tensor-core, packed FP32) once on the caller's own buffers -- all produce the
 * same C -- synchronising the stream, and caches the fastest in the context; later calls of
 * that class use the cached choice without timing.  Inside a stream capture an untuned class
 * takes the fixed rule without timing and without caching it.  With tuning disabled AUTO uses
 * a fixed rule measured on GB300.
 * fp_ctx_autotune_choice reports the cached algorithm for (p, m, n, k) or -1.
 * fp_ctx_autotune errors: FP_EINVAL (ctx NULL). */
fp_status fp_ctx_autotune(fp_ctx ctx, int enable);

/* The cached AUTO choice for (p, m, n, k), or -1 when that class has not been tuned (no
 * counterpart in the paper).  Errors: FP_EINVAL (null ctx or algo). */
fp_status fp_ctx_autotune_choice(fp_ctx ctx, uint32_t p, int m, int n, int k, int* algo);

/* ---------------------------------------------------------------- planner (host only) */

/* Choose packing parameters for products of two polynomials with k coefficients each,
 * n_accum of them summed per result word, in words of type `word`.
 * Rule (Theorem of Sec. 2.3, Eq. bounds, strict reading): q = 2^b is the smallest power of
 * two with q > n_accum * k * (p-1)^2; ndig = 2k-1; the largest possible packed result,
 * sum_j n_accum * min(j+1, 2k-1-j, k) (p-1)^2 q^j, must fit the word's exact range.
 * Errors: FP_EINVAL (p not prime / out of range, k == 0, n_accum == 0, null out),
 * FP_EBOUND (no q fits the word).  Pure host computation: no device needed. */
fp_status fp_dqt_choose(uint32_t p, uint32_t k, uint64_t n_accum, uint32_t word,
                        fp_dqt_params* out);

/* Compression parameters of the right-compressed product (Sec. 7.2-7.4 and 7.6.1) for an
 * inner dimension kdim: Q = 2^b the smallest power of two with kdim (p-1)^2 < Q (Eq. lower,
 * strict), e = the largest number of residues per word whose largest packed value fits the
 * word (Eq. upper; e = floor(beta / log2 Q) up to the exact-range refinement).  For FP32
 * words the inner dimension is chunked: *chunk receives the chunk length (kdim when no
 * chunking is needed) and b, e refer to one chunk.  For FP_MM_SPLIT_F64 (Sec. 7.6) e is the
 * largest compression that pieces of at least min(kdim, 256) entries keep, *chunk the
 * balanced piece length (a multiple of 4, or kdim when one piece suffices) and b that of a
 * piece; for FP_MM_FULL_F64 e = dq1 dt1 and *chunk the piece (fp_mm_full_choose).  Host only.
 * Errors: FP_EINVAL (null outputs, p not a prime <= 251, kdim = 0), FP_EBOUND (no packing
 * fits the algo's word, or the algo's own limit on p). */
fp_status fp_mm_choose(uint32_t p, uint64_t kdim, uint32_t algo, uint32_t* b, uint32_t* e,
                       uint32_t* chunk);

/* Full-compression parameters (Sec. 7.5): Q = 2^b with k' (p-1)^2 < Q for the piece length k'
 * (Eq. lower, strict), dq1 = d_q + 1 rows per left word and dt1 = d_theta + 1 columns per right
 * word, Theta = Q^dq1 (Eq. qtheta), the largest dq1 dt1 (then the most balanced) with
 * dq1, dt1 >= 2 whose largest packed product, dq1 dt1 digits of at most k' (p-1)^2, is below
 * 2^52 (Eq. dq with the exact range of FP64 words and FDIV case 3); *piece = k' (= kdim when the
 * inner dimension is not split; otherwise pieces of at most 4 * ceil(k'/4) entries, balanced,
 * with k' >= min(kdim, 256) where such pieces allow a 2 x 2 packing, else k' >= 16).  Host only.
 * Errors: FP_EINVAL (null outputs, p not a prime <= 251, kdim outside [1, 2^30]), FP_EBOUND (no
 * 2 x 2 packing fits even pieces of 16, i.e. 16 (p-1)^2 >= 2^13: p > 23). */
fp_status fp_mm_full_choose(uint32_t p, uint64_t kdim, uint32_t* b, uint32_t* dq1, uint32_t* dt1,
                            uint32_t* piece);

/* ---------------------------------------------------------------- DQT pack / unpack */

/* DQT (Eq. dqt): words[i] = sum_{j<k} coeffs[i*k + j] * q^j, for i < count, with q = 2^b or
 * q = p 2^b (prm->qform; b <= 32, and p 2^b < 2^40 for the second form).
 * coeffs: device uint8 [count][k] with entries in [0, p-1]; words: device array of count
 * words of type prm->word (double, uint64_t, float or uint32_t).  prm->k <= 64 and
 * (p-1) * sum_j q^j must fit the word (else FP_EBOUND); qform other than the two forms:
 * FP_EINVAL. */
fp_status fp_dqt_pack(fp_ctx ctx, const fp_dqt_params* prm, const uint8_t* coeffs, void* words,
                      size_t count, void* stream);

/* Inverse DQT by REDQ (Algorithm 2 with the FDIV division of Sec. 4 and tabulated
 * correction, Sec. 3.5): coeffs[i*ndig + j] = (j-th base-q digit of words[i]) mod p, where
 * the top digit (j = ndig-1) takes all remaining high bits.  Each word must be a
 * non-negative integer < the word's exact range (2^52 for F64, 2^23 for F32) whose lower
 * ndig-1 base-q digits are < q -- which holds whenever it was produced under the planner's
 * bounds.  With qform = FP_Q_P_POW2 (q = p 2^b, the conclusion's alternative) the compression
 * takes floor(r / p^(i+1)) by ndig successive FDIV divisions by p, floor(r / q^i) as
 * floor(r / p^i) >> (b i), and needs no correction step (p | q, Theorem REDQ).
 * words: device [count] of prm->word; coeffs: device uint8 [count][ndig].
 * Errors: FP_EINVAL (ctx or arrays NULL; p, word, b, qform or ndig out of range), FP_ECUDA. */
fp_status fp_dqt_unpack_redq(fp_ctx ctx, const fp_dqt_params* prm, const void* words,
                             uint8_t* coeffs, size_t count, void* stream);

/* ---------------------------------------------------------------- polynomial product */

/* Batched product over F_p[X] (Sec. 5): for each of `batch` pairs, C = A * B mod p.
 * A: device uint8 [batch][dega+1], B: [batch][degb+1], C: [batch][dega+degb+1], coefficients
 * lowest degree first.  DQT algos pack each operand in one word when the product fits one
 * word, else split into blocks of d+1 coefficients (FQT, Sec. 5.2) and accumulate the block
 * products in words before one REDQ per result block.  FP_ALGO_KARATSUBA forms the same
 * block-product words by Karatsuba splitting of the word polynomials (zero-padded to m 2^L
 * words, 3^L leaf products, exact in Z/2^64 since every result word is below 2^64 under the
 * FQT bound) and then reduces them the same way.  dega, degb <= 1023.
 * Errors: FP_EINVAL, FP_EBOUND (a forced word type cannot hold even d = 0). */
fp_status fp_polymul_batched(fp_ctx ctx, uint32_t p, const uint8_t* A, uint32_t dega,
                             const uint8_t* B, uint32_t degb, uint8_t* C, size_t batch, int algo,
                             void* stream);

/* Kernels of fp_polymul_batched. */
enum { FP_PM_SINGLE_WORD = 0, FP_PM_FQT = 1, FP_PM_KARATSUBA = 2, FP_PM_PLAIN = 3 };

/* The representation fp_polymul_batched runs in for these degrees and this algo. */
typedef struct {
  uint32_t kernel;        /* FP_PM_* */
  uint32_t word;          /* fp_word of the packed words (unused for FP_PM_PLAIN) */
  uint32_t blk_a, blk_b;  /* coefficients per packed word of A and of B: dega+1 and degb+1 for
                             one word per operand, d+1 for the FQT forms */
  uint32_t b;             /* q = 2^b */
  uint32_t ndig;          /* residues per result word: dega+degb+1, or 2d+1 for the FQT forms */
  uint32_t L, m;          /* Karatsuba FQT: split depth and leaf length in words (0 otherwise) */
} fp_polymul_plan_t;

/* Host query of the planner (no device work; Eq. bounds with the exact largest packed value,
 * Sec. 5.2 for the block size): the plan fp_polymul_batched follows for (p, dega, degb, algo).
 * Errors: FP_EINVAL (arguments as in fp_polymul_batched), FP_EBOUND (as fp_polymul_batched). */
fp_status fp_polymul_plan(uint32_t p, uint32_t dega, uint32_t degb, int algo, fp_polymul_plan_t* out);

/* ---------------------------------------------------------------- dot product */

/* Modular dot product (Algorithm 1 with degree-0 entries): *out = (sum u_i v_i) mod p.
 * u, v: device uint8 [n]; out: device uint32 scalar.  DQT algos use the middle-product
 * packing of Sec. 7.1 (d+1 entries per word, reversed on the left), PLAIN uses delayed
 * reduction.  n <= 2^40.  Uses context scratch for per-block partial results.
 * Errors: FP_EINVAL (ctx, out or arrays NULL, p not a prime <= 251, n > 2^40, bad algo;
 * a residue >= p is reported by fp_ctx_status), FP_EBOUND (a forced packing does not fit). */
fp_status fp_dot(fp_ctx ctx, uint32_t p, const uint8_t* u, const uint8_t* v, size_t n,
                 uint32_t* out, int algo, void* stream);

/* Allocation-free variant of fp_dot (the paper has no counterpart: this is an interface for
 * callers that cannot allocate device memory, e.g. code running under an allocator owned by
 * someone else, or a real-time path where cudaMalloc's implicit synchronisation and failure
 * modes are not allowed).  It needs no context and calls no cudaMalloc / cudaFree.  Its
 * scratch (per-block partial sums plus one error word, FP_DOT_NOALLOC_MAX_PARTIALS slots) is a
 * fixed array in the library's device image, present on every GPU that loads the library
 * until the process exits.  The first call on each device looks up that array's device
 * address (with the device current); make that first call before any stream capture.
 * All calls on a device share the array: calls whose work overlaps on the GPU (different
 * streams without ordering) race and may return wrong results.  *out = (sum u_i v_i) mod p,
 * or 0xFFFFFFFF if an input residue was outside [0, p-1].  n <= 2^40 (FP_EINVAL beyond);
 * FP_EUNSUPPORTED if the device would need more partial slots than the array holds. */
#define FP_DOT_NOALLOC_MAX_PARTIALS 4096
fp_status fp_dot_noalloc(uint32_t p, const uint8_t* u, const uint8_t* v, size_t n, uint32_t* out,
                         int algo, void* stream);

/* ---------------------------------------------------------------- matrix product */

/* C = A * B mod p (Sec. 7).  A: device uint8 m x k (leading dimension lda >= k), B: k x n
 * (ldb >= n), C: m x n (ldc >= n).  m, n, k in [1, 2^20]; k also bounded by the algorithm's
 * exactness rule (FP_EBOUND beyond it: e.g. PLAIN_TC needs k (p-1)^2 < 2^24).  Packed
 * algorithms keep the compressed B (k x ceil(n/e) words) in context scratch. */
fp_status fp_matmul(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                    const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, void* stream);

/* One product of a group (see fp_matmul_grouped); fields as in fp_matmul. */
typedef struct {
  uint32_t p;
  int m, n, k;
  const uint8_t* A;
  int lda;
  const uint8_t* B;
  int ldb;
  uint8_t* C;
  int ldc;
} fp_mm_problem;

/* Problems per persistent launch of fp_matmul_grouped. */
#define FP_GROUP_MAX 16

/* Several independent products C_i = A_i B_i mod p_i (the paper has no counterpart: it treats
 * one product at a time; this call schedules Sec. 7's plain product, with the delayed
 * reduction of Sec. 2.2, over many of them).  `problems` is a HOST array of `count` entries
 * (count = 0 is a no-op); every entry is checked as fp_matmul checks its arguments, including
 * the forced algorithm's exactness rule (FP_EBOUND), before anything is enqueued.  Output ranges must not overlap one another or any input.
 * With algo FP_MM_AUTO or FP_MM_PLAIN_F8, the problems with p <= 17, k (p-1)^2 < 2^24, A and
 * B 16-byte aligned and lda, ldb multiples of 16 run together in persistent tensor-core
 * launches of up to FP_GROUP_MAX problems: one CTA per SM takes 128 x 256 output tiles from
 * all of them (longest inner dimension first), its epilogue overlapping the next tile's
 * multiplications; the residue bytes are read in place as e4m3 operands.  Every other problem
 * runs through fp_matmul with the same algo, in order, on the same stream.  Residues >= p set
 * the context's range error (fp_ctx_status).  With algo FP_MM_RIGHT_TC (packed fp16, two
 * residues of C per MMA column, Sec. 7.4) or FP_MM_PLAIN_TC (bf16) every problem runs in the
 * persistent 16-bit kernel's grouped launches, after a conversion of each A and B into
 * context scratch. */
fp_status fp_matmul_grouped(fp_ctx ctx, const fp_mm_problem* problems, size_t count, int algo,
                            void* stream);

/* Right compression of B alone (Sec. 7.4): CB[l][j] = sum_{t<e} B[l][j e + t] Q^t with
 * Q = 2^b, missing columns of the last block taken as zero (partial compression, Sec. 7.1).
 * CB: device array k x ceil(n/e) of `word` (F64 or F32 or U64).  Exposed for tests and reuse.
 * Errors: FP_EINVAL (sizes, b, e or word out of range), FP_EBOUND (the packed word
 * exceeds the word's exact range). */
fp_status fp_pack_cb(fp_ctx ctx, uint32_t p, int k, int n, const uint8_t* B, int ldb,
                     uint32_t b, uint32_t e, uint32_t word, void* CB, void* stream);

/* ---------------------------------------------------------------- GF(p^k) */

/* Build GF(p^k) (Sec. 6): p prime <= 251, k >= 1, p^k <= 65536.  The modulus is the monic
 * irreducible of degree k with the smallest key sum_{i<k} c_i p^i (brute-force
 * irreducibility test); q = 2^b is the smallest power of two above k (p-1)^2; the tables of
 * Algorithm FGDP (element -> packed word, L and H folding the REDQ correction and the
 * reduction by the modulus) are built on the host and copied to the device.  Elements are
 * indices sum_i c_i p^i: uint8 when p^k <= 256, else uint16.
 * Errors: FP_EINVAL (p, k or p^k out of range), FP_EUNSUPPORTED (tables or the product
 * word too large), FP_ENOMEM, FP_ECUDA. */
fp_status fp_gf_create(fp_ctx ctx, uint32_t p, uint32_t k, fp_gf* out);

/* Free a field's host and device tables (NULL ok).  Resource management: no counterpart in
 * the paper. */
void fp_gf_destroy(fp_gf gf);

/* Query a field (Sec. 6, the parameters of Algorithm FGDP's tables): modulus coefficients
 * (k+1 values, constant term first) into `modulus` (may be NULL), q exponent b, packed word
 * type, and element width in bytes.  Errors: FP_EINVAL (gf NULL). */
fp_status fp_gf_info(fp_gf gf, uint32_t* modulus, uint32_t* b, uint32_t* word,
                     uint32_t* elem_bytes);

/* Batched multiply c[i] = a[i] * b[i] in GF(p^k) by Algorithm FGDP with n = 1: table DQT,
 * one word product, REDQ compression, two lookups (L, H) and one field addition.
 * a, b, c: device arrays of `count` element indices (width per fp_gf_info).
 * Errors: FP_EINVAL (null ctx, field or arrays; an index >= p^k is reported by
 * fp_ctx_status). */
fp_status fp_gf_mul_batched(fp_ctx ctx, fp_gf gf, const void* a, const void* b, void* c,
                            size_t count, void* stream);

/* Element forms of fp_gf_dot.  FP_GF_LOG is the discrete-log form Algorithm FGDP assumes:
 * the element g^e is written e (0 <= e <= p^k - 2) and zero is written p^k - 1, where g is
 * the smallest index of multiplicative order p^k - 1 (fp_gf_dot_info). */
enum { FP_GF_INDEX = 0, FP_GF_LOG = 1 };

/* Dot product over GF(p^k) by Algorithm FGDP (Sec. 6): *out = sum_i a[i] b[i] in the field.
 * a, b: device arrays of n elements in `form` (width per fp_gf_info); out: one device element
 * of the same width, written in the same form.  The conversion to words is one table lookup
 * from either form to the element's evaluation at the dot product's own q = 2^b_dot; the word products
 * accumulate for `chunk` terms (every digit below q, the word below 2^64) before each REDQ and
 * L/H lookup, and the partial results are added in the field.  GF(3^5), GF(7^4) and GF(2^8)
 * with 16-byte aligned arrays (either form) run on 32-bit words with REDQ in SWAR form:
 * GF(3^5) at q = 2^7 with six products per REDQ, GF(7^4) at q = 2^9 with three, and GF(2^8) at
 * q = 2^4 with the word products XOR-accumulated and one REDQ per thread (p | q: the
 * compression values are the digits' lowest bits, which XOR adds mod 2).  n = 0 writes
 * zero.  Codes >= p^k set FP_EINVAL on the context (read by fp_ctx_status) and count as zero.
 * n < 2^40.
 * Uses context scratch for per-block partial sums. */
fp_status fp_gf_dot(fp_ctx ctx, fp_gf gf, const void* a, const void* b, size_t n, void* out,
                    int form, void* stream);

/* Matrix product over GF(p^k) by Algorithm FGDP (Sec. 6) on every entry: C = A B in the field,
 * C[r][c] = sum_l A[r][l] B[l][c].  A: device m x k elements (leading dimension lda >= k), B:
 * k x n (ldb >= n), C: m x n (ldc >= n), all in `form` (index or discrete log, width per
 * fp_gf_info), leading dimensions in elements.  Each element is converted once per use tile by
 * the dot product's word table (q = 2^b_dot of fp_gf_dot_info), word products accumulate for
 * `chunk` inner steps before each REDQ and L/H lookup, and the partial results are added in the
 * field; GF(3^5), GF(7^4) and GF(2^8) take the 32-bit word forms of fp_gf_dot.
 * m, n, k in [1, 2^20].  Codes >= p^k set FP_EINVAL on the context (fp_ctx_status) and
 * count as zero.  Errors: FP_EINVAL (null ctx, field or arrays; sizes or leading dimensions),
 * FP_EUNSUPPORTED (the field's tables do not fit one block's shared memory), FP_ECUDA. */
fp_status fp_gf_matmul(fp_ctx ctx, fp_gf gf, int m, int n, int k, const void* A, int lda, const void* B,
                       int ldb, void* C, int ldc, int form, void* stream);

/* The dot product's parameters (Algorithm FGDP, Sec. 6): index of the generator g of the log
 * form, exponent b_dot of its q, and the number of word products accumulated per REDQ, as the
 * general 64-bit word path uses them (the 32-bit word forms of GF(3^5), GF(7^4), GF(2^8) fix
 * their own, stated at fp_gf_dot).  Any output may be NULL.  Errors: FP_EINVAL (gf NULL). */
fp_status fp_gf_dot_info(fp_gf gf, uint32_t* generator, uint32_t* b_dot, uint32_t* chunk);

/* ---------------------------------------------------------------- uneven batches */

/* One instance of an uneven batch: kind 0 = matmul (C = A B mod p, dense row-major,
 * A m x k, B k x n, C m x n), kind 1 = dot (n = 1, m = 1, A = u[k], B = v[k], C = uint32
 * result stored as 4 bytes).  All pointers are device pointers owned by the caller. */
typedef struct {
  uint32_t kind;
  uint32_t p;
  uint32_t m, n, k;
  uint32_t reserved;
  const uint8_t* A;
  const uint8_t* B;
  uint8_t* C;
} fp_instance;

/* Uneven batch (no counterpart in the paper as a call; each instance's packing follows
 * Sec. 7.6.1).  Runs all `count` instances, routed by size:
 *  - matrix products with p <= 17 and k (p-1)^2 < 2^23, or p <= 31 and 2 k (p/2)^2 + p < 2^23,
 *    whose sizes rounded up to 128 x 256 x 32 blocks give >= 2^21 MACs and at most 32 times
 *    their own (or any such with k >= 128): the e4m3 tensor-core kernel.  One launch first lays
 *    every such operand out as swizzled 16 KB tiles (residues range-checked and, in the second
 *    case, centred to |c| <= p/2), then one persistent launch takes up to 4096 products; any
 *    row stride and alignment of the caller's arrays;
 *  - those with 31 < p <= 127, m, n >= 64, m n k >= 2^21 and k (p-1)^2 < 2^24: the bf16 kernel
 *    (operands converted and range-checked in one launch, up to 64 products per launch);
 *  - everything else: ONE persistent kernel launch whose CTAs take tiles from a device work
 *    queue (an atomic counter over a tile list the host planner sorts by cost), packing degree
 *    e and word chosen per (p, k) by the planner and the autotuner cache in the context.
 * `instances` is a HOST array; every instance is checked before anything is enqueued; the
 * plan is copied to context scratch through pinned staging (the call does not wait for earlier
 * work on the stream).  Stream capture: a call captured into a CUDA graph writes its plan with
 * kernels whose parameters carry it (so each replay runs the captured batch even after other
 * calls), takes the packing degree from the tuning cache or the fixed rule, and refuses with
 * FP_EUNSUPPORTED if it would have to grow context scratch -- make the same call once outside
 * the capture first.  Scratch a captured graph used is not freed before fp_ctx_destroy; replays
 * and other calls on the context must be ordered on one stream (they share that scratch).
 * Errors: FP_EINVAL, FP_EBOUND, FP_ECUDA, FP_ENOMEM, FP_EUNSUPPORTED. */
fp_status fp_batch_run(fp_ctx ctx, const fp_instance* instances, size_t count, void* stream);

/* Diagnostic (no counterpart in the paper): launches one warp that waits on a device barrier
 * nothing will complete, using the library's bounded wait with a limit of `polls` polls
 * (1 <= polls <= 2^22).  The wait gives up, the context's sticky flag records the timeout and
 * the next fp_ctx_status returns FP_ETIMEOUT; the GPU context stays usable.  Exercises the
 * failure path the tensor-core kernels take if a TMA or MMA completion never arrives. */
fp_status fp_selftest_bounded_wait(fp_ctx ctx, uint32_t polls, void* stream);

/* ---------------------------------------------------------------- serving loop */

/* A request for the serving loop.  kind: 0 polymul (a = dega, b = degb, p), 1 dot (a = n, p),
 * 2 GF(p^k) batch multiply (a = count, gf), 3 matmul (a = m, b = n, c = k, p).  Inputs are
 * HOST buffers (pinned memory recommended) laid out as for the corresponding call (polymul:
 * A[dega+1], B[degb+1]; dot: u[n], v[n]; GF: a[count], b[count] element indices; matmul:
 * A m x k, B k x n, dense); host_out receives the result (polymul dega+degb+1 bytes, dot a
 * uint32, GF count indices, matmul m x n bytes).  The caller keeps all three buffers alive
 * until the request is reported done. */
typedef struct {
  uint32_t kind;
  uint32_t p;
  uint32_t a, b, c;
  uint32_t reserved;
  fp_gf gf;
  const void* host_a;
  const void* host_b;
  void* host_out;
} fp_request;

/* arena_bytes: device memory for the buffers of in-flight requests (admission budget);
 * streams: CUDA streams whose batches may overlap on the GPU; max_batch: requests per batch;
 * window_us: while the GPU is busy, how long a forming batch may wait to grow. */
typedef struct {
  uint64_t arena_bytes;
  uint32_t streams;
  uint32_t max_batch;
  uint32_t window_us;
  uint32_t reserved;
} fp_server_config;

typedef struct {
  uint64_t submitted, completed, batches, launches, failed;
} fp_server_stats;

typedef struct fp_server_s* fp_server;

/* Continuous batching (no counterpart in the paper; the systems layer around the packed
 * kernels): a scheduler thread takes submitted requests in arrival order, admits them as
 * arena memory frees up, packs every admitted request into one batch (gathered host-to-device
 * copy, one launch per request kind: varlen blocked-FQT polymul, segmented GF multiply, the
 * persistent matmul/dot kernel of fp_batch_run, and for matmul requests with p <= 17, m, n >= 64,
 * k (p-1)^2 < 2^24 and m n k >= 2^21 the grouped e4m3 tensor-core kernel of fp_matmul_grouped
 * (their rows staged at 16-byte strides); one device-to-host copy), issues batches
 * round-robin on its streams so that new batches start while earlier ones run, and records
 * each request's latency (submission to observed completion, host steady clock).
 * Errors: FP_EINVAL (bad config), FP_ENOMEM, FP_ECUDA. */
fp_status fp_server_create(fp_ctx ctx, const fp_server_config* cfg, fp_server* out);

/* Serving (no counterpart in the paper).  Thread-safe.  Validates the request (FP_EINVAL,
 * FP_EBOUND) and queues it; *ticket numbers requests from 0 in submission order. */
fp_status fp_server_submit(fp_server s, const fp_request* req, uint64_t* ticket);

/* Serving (no counterpart in the paper).  Thread-safe.  Submits the n requests of the host
 * array `reqs` (the caller's array; read during the call only): every request is validated
 * first, and if one fails (FP_EINVAL, FP_EBOUND, message naming it) none is queued; else all
 * are queued, in order, with tickets *first_ticket .. *first_ticket + n - 1 and one submission
 * time.  Errors: FP_EINVAL (null server, array or output), FP_EBOUND. */
fp_status fp_server_submit_many(fp_server s, const fp_request* reqs, size_t n, uint64_t* first_ticket);

/* Serving (no counterpart in the paper): *done = 1 once the result is in host_out (then
 * *latency_us is set), else 0.  A request that failed on the device reports done = -1.
 * Errors: FP_EINVAL (null server or outputs, unknown ticket). */
fp_status fp_server_poll(fp_server s, uint64_t ticket, int* done, double* latency_us);

/* Serving (no counterpart in the paper): wait until every submitted request is done.
 * Errors: FP_ETIMEOUT when timeout_s passes first, FP_EINVAL (null server). */
fp_status fp_server_drain(fp_server s, double timeout_s);

/* Serving (no counterpart in the paper): latencies in microseconds of tickets
 * [first, first+n) into out; -1 for a ticket not done, failed or not yet issued.
 * Errors: FP_EINVAL (null server or out). */
fp_status fp_server_latencies(fp_server s, uint64_t first, size_t n, double* out);

/* Serving (no counterpart in the paper): counters of submitted, completed and failed
 * requests, batches and kernel launches.  Errors: FP_EINVAL (null). */
fp_status fp_server_stats_get(fp_server s, fp_server_stats* out);

/* Serving (no counterpart in the paper): stops the scheduler after draining outstanding work
 * (bounded) and frees everything.  NULL ok. */
void fp_server_destroy(fp_server s);

#ifdef __cplusplus
}
#endif
#endif /* FPDQT_H */
