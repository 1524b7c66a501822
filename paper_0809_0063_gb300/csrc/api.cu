// C ABI entry points of libfpdqt: context, errors, planner (Sec. 2.3, 7.2, 7.6.1) and the
// argument checks in front of every kernel launcher.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <cstring>

#include "fpdqt_internal.cuh"

namespace fpd {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

fp_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %s (%d) in %s", cudaGetErrorString(e), (int)e, what);
  return FP_ECUDA;
}

bool is_prime(uint32_t p) {
  if (p < 2) return false;
  for (uint32_t d = 2; d * d <= p; ++d)
    if (p % d == 0) return false;
  return true;
}

DivP make_divp(uint32_t p) {
  DivP d{};
  uint32_t l = 0;
  while ((1ull << l) < p) ++l;
  d.l = l;
  d.pow2 = (p & (p - 1)) == 0;
  d.sh = 0;
  if (d.pow2) {
    while ((1u << d.sh) < p) ++d.sh;
    return d;
  }
  unsigned __int128 two_l = (unsigned __int128)1 << l;
  unsigned __int128 m64 = (((unsigned __int128)1 << 64) * (two_l - p)) / p + 1;
  d.m64 = (uint64_t)m64;
  uint64_t m32 = ((((uint64_t)1) << 32) * ((1ull << l) - p)) / p + 1;
  d.m32 = (uint32_t)m32;
  return d;
}

int word_beta(uint32_t word) {
  switch (word) {
    case FP_WORD_F64: return 52;
    case FP_WORD_U64: return 64;
    case FP_WORD_F32: return 23;
    case FP_WORD_U32: return 32;
    default: return 0;
  }
}

size_t word_bytes(uint32_t word) {
  return (word == FP_WORD_F64 || word == FP_WORD_U64) ? 8 : 4;
}

// Round-up reciprocals by the exact-residual test: fma(x, p, -1) is the exact sign of
// x p - 1, so x < 1/p exactly when it is negative, and then the next float up is RU(1/p).
static double ru_recip_d(uint32_t p) {
  double x = 1.0 / (double)p;
  if (fma(x, (double)p, -1.0) < 0.0) x = nextafter(x, INFINITY);
  return x;
}
static float ru_recip_f(uint32_t p) {
  float x = 1.0f / (float)p;
  if (fmaf(x, (float)p, -1.0f) < 0.0f) x = nextafterf(x, INFINITY);
  return x;
}

RedqParams make_redq(uint32_t p, uint32_t b, uint32_t ndig) {
  RedqParams P{};
  P.p = p;
  P.b = b;
  P.ndig = ndig;
  uint64_t qmodp = (b >= 64) ? 0 : ((1ull << b) % p);
  P.c = (uint32_t)((p - qmodp) % p);
  if (qmodp == 0) P.mode = CORR_NONE;
  else if (p * p * p <= 32) P.mode = CORR_SHFL3;
  else if (p * p <= 32) P.mode = CORR_SHFL2;
  else if (p <= 31) P.mode = CORR_SMEM2;
  else P.mode = CORR_ARITH;
  P.invp_d = ru_recip_d(p);
  P.invp_f = ru_recip_f(p);
  P.dv = make_divp(p);
  return P;
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();   // a query that failed leaves no sticky error behind
    return false;
  }
  return cs == cudaStreamCaptureStatusActive;
}

fp_status ensure_scratch(fp_ctx ctx, size_t bytes, int which, cudaStream_t st) {
  void** ptr = which ? &ctx->scratch2 : &ctx->scratch;
  size_t* cap = which ? &ctx->scratch2_bytes : &ctx->scratch_bytes;
  const bool capturing = stream_capturing(st);
  if (*cap >= bytes) {
    if (capturing) ctx->captured = true;   // a graph now refers to this buffer
    return FP_OK;
  }
  FP_CHECK(!capturing, FP_EUNSUPPORTED,
           "this call needs %zu bytes of context scratch during a stream capture (%zu held): make the same "
           "call once outside the capture first", bytes, *cap);
  if (*ptr) {
    if (ctx->captured) {
      ctx->retired.push_back(*ptr);          // a captured graph may still use it: freed with the context
    } else {
      FP_CUDA(cudaDeviceSynchronize());
      FP_CUDA(cudaFree(*ptr));
    }
    *ptr = nullptr;
    *cap = 0;
  }
  size_t want = bytes < (1u << 20) ? (1u << 20) : bytes + bytes / 8;
  cudaError_t e = cudaMalloc(ptr, want);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    set_error("cudaMalloc of %zu bytes of scratch failed: %s", want, cudaGetErrorString(e));
    return FP_ENOMEM;
  }
  *cap = want;
  return FP_OK;
}

// Bytes written to device memory by kernels whose parameters carry them: the form of an upload
// that a stream capture records by value (a captured copy from pinned host memory would read
// the staging buffer again at every replay, after later calls had rewritten it).
struct InlineChunk {
  static constexpr uint32_t CAP = 32000;   // the parameter block stays under the 32 KB limit
  uint32_t n;
  uint8_t b[CAP];
};

// One 4-byte word per thread over as many CTAs as the chunk needs: kernel parameters are read
// through the constant cache, which serves one address per cycle, so one CTA reading a whole
// chunk (a byte per load) took ~19 us per chunk; spread over CTAs (one SM's cache each) and read
// by words it takes a few.
__global__ void k_put_bytes(uint8_t* __restrict__ dst, const __grid_constant__ InlineChunk c) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nw = c.n / 4;
  if ((((uintptr_t)dst) & 3u) == 0) {
    if (i < nw) reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(c.b)[i];
    if (i < c.n - 4 * nw) dst[4 * nw + i] = c.b[4 * nw + i];
  } else {
    for (uint32_t j = i; j < c.n; j += gridDim.x * blockDim.x) dst[j] = c.b[j];
  }
}

static fp_status upload_inline(fp_ctx ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  static InlineChunk c;   // host-side parameter block, copied into each launch
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  for (size_t off = 0; off < bytes; off += InlineChunk::CAP) {
    c.n = (uint32_t)std::min<size_t>(InlineChunk::CAP, bytes - off);
    std::memcpy(c.b, (const uint8_t*)src + off, c.n);
    const int grid = (int)((c.n / 4 + 255) / 256) + 1;
    FP_LAUNCH(ctx, "k_put_bytes", st, k_put_bytes<<<grid, 256, 0, st>>>((uint8_t*)dst + off, c));
    FP_CUDA(cudaGetLastError());
  }
  return FP_OK;
}

fp_status upload_staged(fp_ctx ctx, int slot, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return FP_OK;
  if (stream_capturing(st)) return upload_inline(ctx, dst, src, bytes, st);
  if (ctx->pin_ev[slot]) FP_CUDA(cudaEventSynchronize(ctx->pin_ev[slot]));
  else FP_CUDA(cudaEventCreateWithFlags(&ctx->pin_ev[slot], cudaEventDisableTiming));
  if (ctx->pin_bytes[slot] < bytes) {
    if (ctx->pin[slot]) FP_CUDA(cudaFreeHost(ctx->pin[slot]));
    ctx->pin[slot] = nullptr;
    ctx->pin_bytes[slot] = 0;
    const size_t want = bytes < (1u << 16) ? (1u << 16) : bytes + bytes / 4;
    FP_CUDA(cudaMallocHost(&ctx->pin[slot], want));
    ctx->pin_bytes[slot] = want;
  }
  std::memcpy(ctx->pin[slot], src, bytes);
  FP_CUDA(cudaMemcpyAsync(dst, ctx->pin[slot], bytes, cudaMemcpyHostToDevice, st));
  FP_CUDA(cudaEventRecord(ctx->pin_ev[slot], st));
  return FP_OK;
}

// Largest packed value when n_accum products of two k-coefficient polynomials with entries
// in [0, p-1] are summed: digit j collects n_accum * min(j+1, 2k-1-j, k) products.
static bool poly_word_fits(uint32_t p, uint32_t k, uint64_t n_accum, uint32_t b, int beta) {
  unsigned __int128 total = 0;
  unsigned __int128 lim = ((unsigned __int128)1 << beta);  // values must be < 2^beta
  uint32_t nd = 2 * k - 1;
  for (uint32_t j = 0; j < nd; ++j) {
    uint64_t terms = j + 1;
    if (nd - j < terms) terms = nd - j;
    if (k < terms) terms = k;
    unsigned __int128 dig = (unsigned __int128)n_accum * terms * (uint64_t)(p - 1) * (p - 1);
    if ((uint64_t)j * b >= 128) return dig == 0;
    unsigned __int128 sh = dig << (j * b);
    if ((sh >> (j * b)) != dig) return false;
    total += sh;
    if (total >= lim) return false;
  }
  return total < lim;
}

static cudaEvent_t pool_get(fp_ctx ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void launch_begin(fp_ctx ctx, const char* name, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->pmu);
  ctx->launches++;
  if (!ctx->prof) return;
  fp_ctx_s::Rec r{name, pool_get(ctx), pool_get(ctx)};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  ctx->recs.push_back(r);
}

void launch_end(fp_ctx ctx, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->pmu);
  if (!ctx->prof || ctx->recs.empty()) return;
  cudaEventRecord(ctx->recs.back().b, st);
}

}  // namespace fpd

using namespace fpd;

// ------------------------------------------------------------------ instrumentation

extern "C" fp_status fp_ctx_profile(fp_ctx ctx, int mode) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_ctx_profile: ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->pmu);
  if (mode == 2) {
    for (auto& r : ctx->recs) {
      cudaEventSynchronize(r.b);
      ctx->pool.push_back(r.a);
      ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    return FP_OK;
  }
  FP_CHECK(mode == 0 || mode == 1, FP_EINVAL, "fp_ctx_profile: mode must be 0, 1 or 2");
  ctx->prof = mode;
  return FP_OK;
}

extern "C" fp_status fp_ctx_profile_read(fp_ctx ctx, const char* prefix, uint64_t* launches, double* total_ms) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_ctx_profile_read: ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->pmu);
  uint64_t n = 0;
  double ms = 0;
  size_t pl = prefix ? strlen(prefix) : 0;
  for (auto& r : ctx->recs) {
    if (pl && strncmp(r.name, prefix, pl) != 0) continue;
    FP_CUDA(cudaEventSynchronize(r.b));
    float t = 0;
    FP_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return FP_OK;
}

extern "C" fp_status fp_ctx_launches(fp_ctx ctx, uint64_t* count) {
  FP_CHECK(ctx && count, FP_EINVAL, "fp_ctx_launches: null argument");
  std::lock_guard<std::mutex> lk(ctx->pmu);
  *count = ctx->launches;
  return FP_OK;
}

// ------------------------------------------------------------------ context

extern "C" fp_status fp_ctx_create(fp_ctx* out, int device) {
  FP_CHECK(out != nullptr, FP_EINVAL, "fp_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  FP_CUDA(cudaGetDeviceCount(&ndev));
  FP_CHECK(device >= 0 && device < ndev, FP_EINVAL, "fp_ctx_create: device %d of %d", device, ndev);
  FP_CUDA(cudaSetDevice(device));
  fp_ctx c = new (std::nothrow) fp_ctx_s();
  FP_CHECK(c != nullptr, FP_ENOMEM, "fp_ctx_create: out of host memory");
  c->device = device;
  cudaDeviceProp pr;
  cudaError_t e = cudaGetDeviceProperties(&pr, device);
  if (e == cudaSuccess) c->num_sms = pr.multiProcessorCount;
  e = cudaMalloc(&c->d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    if (c->d_err) cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "fp_ctx_create");
  }
  *out = c;
  return FP_OK;
}

extern "C" void fp_ctx_destroy(fp_ctx ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->scratch2) cudaFree(ctx->scratch2);
  for (void* x : ctx->retired) cudaFree(x);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  for (int i = 0; i < fp_ctx_s::PIN_SLOTS; ++i) {
    if (ctx->pin[i]) cudaFreeHost(ctx->pin[i]);
    if (ctx->pin_ev[i]) cudaEventDestroy(ctx->pin_ev[i]);
  }
  delete ctx;
}

extern "C" fp_status fp_ctx_status(fp_ctx ctx, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_ctx_status: ctx is NULL");
  FP_CUDA(cudaStreamSynchronize(as_stream(stream)));
  uint32_t h = 0;
  FP_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost));
  FP_CUDA(cudaMemset(ctx->d_err, 0, sizeof h));
  if (h & ERR_TIMEOUT) {
    set_error("a bounded device wait gave up (timeout)");
    return FP_ETIMEOUT;
  }
  if (h & ERR_RANGE) {
    set_error("an input residue or element index was out of range");
    return FP_EINVAL;
  }
  return FP_OK;
}

extern "C" const char* fp_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------ planner

extern "C" fp_status fp_dqt_choose(uint32_t p, uint32_t k, uint64_t n_accum, uint32_t word,
                                   fp_dqt_params* out) {
  FP_CHECK(out != nullptr, FP_EINVAL, "fp_dqt_choose: out is NULL");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "fp_dqt_choose: p=%u is not a prime <= 251", p);
  FP_CHECK(k >= 1 && k <= 64, FP_EINVAL, "fp_dqt_choose: k=%u outside [1, 64]", k);
  FP_CHECK(n_accum >= 1, FP_EINVAL, "fp_dqt_choose: n_accum must be >= 1");
  int beta = word_beta(word);
  FP_CHECK(beta > 0, FP_EINVAL, "fp_dqt_choose: bad word type %u", word);
  // Theorem (Eq. bounds), strict: q > n k (p-1)^2.
  unsigned __int128 bound = (unsigned __int128)n_accum * k * (uint64_t)(p - 1) * (p - 1);
  uint32_t b = 0;
  while (((unsigned __int128)1 << b) <= bound) ++b;
  if (b == 0) b = 1;
  FP_CHECK(poly_word_fits(p, k, n_accum, b, beta), FP_EBOUND,
           "fp_dqt_choose: p=%u k=%u n=%llu needs q=2^%u and %u digits: exceeds %d exact bits",
           p, k, (unsigned long long)n_accum, b, 2 * k - 1, beta);
  out->p = p;
  out->k = k;
  out->b = b;
  out->ndig = 2 * k - 1;
  out->word = word;
  out->qform = FP_Q_POW2;
  out->n_accum = n_accum;
  return FP_OK;
}

namespace fpd {
// Right compression parameters (Sec. 7.2-7.4): see fp_mm_choose in the header.
fp_status mm_choose(uint32_t p, uint64_t kdim, uint32_t algo, uint32_t* b_out, uint32_t* e_out,
                    uint32_t* chunk_out) {
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  if (algo == FP_MM_SPLIT_F64) return split_choose(p, kdim, b_out, e_out, chunk_out);
  if (algo == FP_MM_FULL_F64) {
    uint32_t d1 = 0, t1 = 0;
    const fp_status s = full_choose(p, kdim, b_out, &d1, &t1, chunk_out);
    if (s == FP_OK) *e_out = d1 * t1;
    return s;
  }
  if (algo == FP_MM_RIGHT_F32 || algo == FP_MM_LEFT_F32) {
    // Per chunk: two residues at Qc = 2^12 in one binary32 accumulator; chunk digits
    // kc (p-1)^2 <= 4095 < Qc (Eq. lower, strict) so the word stays <= 4095 * 4097 < 2^24.
    uint32_t kc = pp ? (uint32_t)(4095 / pp) : 4095u;
    kc &= ~7u;  // whole K-steps of the kernel
    if (kc == 0) {
      set_error("RIGHT_F32 needs (p-1)^2 <= 511 (p=%u)", p);
      return FP_EBOUND;
    }
    if ((uint64_t)kc > kdim) kc = (uint32_t)((kdim + 7) & ~7ull);
    *b_out = 12;
    *e_out = 2;
    *chunk_out = kc;
    return FP_OK;
  }
  if (algo == FP_MM_RIGHT_TC) {
    // centred residues {-1,0,1}: |digit| <= chunk < Q/2 with Q = 2^10; fp16 operands hold
    // b0 + 2^10 b1 exactly (11 significant bits).  p = 5, 7: |c| <= (p-1)/2 at Q = 1023 / 681
    // (|c0| + Q |c1| <= 2048, not a power of two: *b = 0), chunks of 64 / 32 inner steps keep
    // |digit| < Q / 2.
    if (p > 3 && p != 5 && p != 7) {
      set_error("RIGHT_TC needs p in {2, 3, 5, 7} (p=%u)", p);
      return FP_EBOUND;
    }
    *b_out = p <= 3 ? 10 : 0;
    *e_out = 2;
    *chunk_out = p <= 3 ? 448 : (p == 5 ? 64 : 32);
    return FP_OK;
  }
  int beta = (algo == FP_MM_RIGHT_F64 || algo == FP_MM_PLAIN_F64 || algo == FP_MM_LEFT_F64) ? 52 : 64;
  unsigned __int128 D = (unsigned __int128)kdim * pp;  // largest digit
  uint32_t b = 1;
  while (((unsigned __int128)1 << b) <= D) ++b;
  unsigned __int128 lim = (unsigned __int128)1 << beta;
  uint32_t e = 0;
  unsigned __int128 total = 0;
  while (true) {
    if ((uint64_t)(e) * b >= 100) break;
    unsigned __int128 nt = total + (D << (e * b));
    if (nt >= lim) break;
    total = nt;
    ++e;
  }
  if (e == 0) {
    set_error("no packing fits: k=%llu p=%u", (unsigned long long)kdim, p);
    return FP_EBOUND;
  }
  if (algo == FP_MM_PLAIN_F64) e = 1;
  *b_out = b;
  *e_out = e;
  *chunk_out = (uint32_t)(kdim > 0xffffffffull ? 0xffffffffu : kdim);
  return FP_OK;
}
}  // namespace fpd

extern "C" fp_status fp_mm_choose(uint32_t p, uint64_t kdim, uint32_t algo, uint32_t* b,
                                  uint32_t* e, uint32_t* chunk) {
  FP_CHECK(b && e && chunk, FP_EINVAL, "fp_mm_choose: null output");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "fp_mm_choose: p=%u not a prime <= 251", p);
  FP_CHECK(kdim >= 1, FP_EINVAL, "fp_mm_choose: kdim must be >= 1");
  return mm_choose(p, kdim, algo, b, e, chunk);
}

// ------------------------------------------------------------------ DQT pack / unpack

static fp_status check_params(const fp_dqt_params* prm, bool pack) {
  FP_CHECK(prm != nullptr, FP_EINVAL, "params is NULL");
  FP_CHECK(prm->p >= 2 && prm->p <= 251 && is_prime(prm->p), FP_EINVAL, "p=%u not a prime <= 251", prm->p);
  int beta = word_beta(prm->word);
  FP_CHECK(beta > 0, FP_EINVAL, "bad word type %u", prm->word);
  FP_CHECK(prm->qform == FP_Q_POW2 || prm->qform == FP_Q_P_POW2, FP_EINVAL, "bad qform %u", prm->qform);
  if (prm->qform == FP_Q_POW2) {
    FP_CHECK(prm->b >= 1 && prm->b <= 32, FP_EINVAL, "b=%u outside [1, 32]", prm->b);
    FP_CHECK((1ull << prm->b) >= prm->p, FP_EINVAL, "q=2^%u below p=%u", prm->b, prm->p);
  } else {
    FP_CHECK(prm->b <= 32 && ((uint64_t)prm->p << prm->b) < (1ull << 40), FP_EINVAL,
             "q=p 2^%u outside [p, 2^40)", prm->b);
  }
  if (pack) {
    FP_CHECK(prm->k >= 1 && prm->k <= 64, FP_EINVAL, "k=%u outside [1, 64]", prm->k);
    // largest packed operand (p-1) sum_{j<k} q^j must be < 2^beta
    const unsigned __int128 lim = (unsigned __int128)1 << beta;
    const unsigned __int128 q = prm->qform == FP_Q_POW2 ? ((unsigned __int128)1 << prm->b)
                                                        : ((unsigned __int128)prm->p << prm->b);
    unsigned __int128 tot = 0, qj = 1;
    for (uint32_t j = 0; j < prm->k; ++j) {
      FP_CHECK(qj < lim, FP_EBOUND, "packed operand exceeds the word");
      tot += (unsigned __int128)(prm->p - 1) * qj;
      qj *= q;
    }
    FP_CHECK(tot < lim, FP_EBOUND, "packing k=%u residues at q=%s2^%u exceeds %d exact bits", prm->k,
             prm->qform == FP_Q_POW2 ? "" : "p ", prm->b, beta);
  } else {
    FP_CHECK(prm->ndig >= 1 && prm->ndig <= 64, FP_EINVAL, "ndig=%u outside [1, 64]", prm->ndig);
  }
  return FP_OK;
}

extern "C" fp_status fp_dqt_pack(fp_ctx ctx, const fp_dqt_params* prm, const uint8_t* coeffs,
                                 void* words, size_t count, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_dqt_pack: ctx is NULL");
  fp_status s = check_params(prm, true);
  if (s != FP_OK) return s;
  if (count == 0) return FP_OK;
  FP_CHECK(coeffs && words, FP_EINVAL, "fp_dqt_pack: null array");
  return launch_pack(ctx, *prm, coeffs, words, count, as_stream(stream));
}

extern "C" fp_status fp_dqt_unpack_redq(fp_ctx ctx, const fp_dqt_params* prm, const void* words,
                                        uint8_t* coeffs, size_t count, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_dqt_unpack_redq: ctx is NULL");
  fp_status s = check_params(prm, false);
  if (s != FP_OK) return s;
  if (count == 0) return FP_OK;
  FP_CHECK(coeffs && words, FP_EINVAL, "fp_dqt_unpack_redq: null array");
  return launch_unpack(ctx, *prm, words, coeffs, count, as_stream(stream));
}

extern "C" fp_status fp_polymul_batched(fp_ctx ctx, uint32_t p, const uint8_t* A, uint32_t dega,
                                        const uint8_t* B, uint32_t degb, uint8_t* C, size_t batch,
                                        int algo, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_polymul_batched: ctx is NULL");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "p=%u not a prime <= 251", p);
  FP_CHECK(dega <= 1023 && degb <= 1023, FP_EINVAL, "degrees must be <= 1023");
  FP_CHECK(algo >= FP_ALGO_AUTO && algo <= FP_ALGO_KARATSUBA, FP_EINVAL, "bad algo %d", algo);
  if (batch == 0) return FP_OK;
  FP_CHECK(A && B && C, FP_EINVAL, "fp_polymul_batched: null array");
  return launch_polymul(ctx, p, A, dega, B, degb, C, batch, algo, as_stream(stream));
}

extern "C" fp_status fp_dot(fp_ctx ctx, uint32_t p, const uint8_t* u, const uint8_t* v, size_t n,
                            uint32_t* out, int algo, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_dot: ctx is NULL");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "p=%u not a prime <= 251", p);
  FP_CHECK(out != nullptr, FP_EINVAL, "fp_dot: out is NULL");
  FP_CHECK(n <= (1ull << 40), FP_EINVAL, "fp_dot: n too large");
  FP_CHECK(algo >= FP_ALGO_AUTO && algo <= FP_ALGO_DQT_U32, FP_EINVAL, "bad algo %d", algo);
  FP_CHECK(n == 0 || (u && v), FP_EINVAL, "fp_dot: null array");
  return launch_dot(ctx, p, u, v, n, out, algo, as_stream(stream));
}

static fp_status check_matmul(uint32_t p, int m, int n, int k, const uint8_t* A, int lda, const uint8_t* B,
                              int ldb, const uint8_t* C, int ldc, int algo) {
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "p=%u not a prime <= 251", p);
  FP_CHECK(m >= 1 && n >= 1 && k >= 1 && m <= (1 << 20) && n <= (1 << 20) && k <= (1 << 20),
           FP_EINVAL, "fp_matmul: sizes m=%d n=%d k=%d outside [1, 2^20]", m, n, k);
  FP_CHECK(lda >= k && ldb >= n && ldc >= n, FP_EINVAL, "fp_matmul: leading dimensions too small");
  FP_CHECK(A && B && C, FP_EINVAL, "fp_matmul: null array");
  FP_CHECK(algo >= FP_MM_AUTO && algo <= FP_MM_SPLIT_F64, FP_EINVAL, "bad algo %d", algo);
  return FP_OK;
}

extern "C" fp_status fp_matmul(fp_ctx ctx, uint32_t p, int m, int n, int k, const uint8_t* A, int lda,
                               const uint8_t* B, int ldb, uint8_t* C, int ldc, int algo, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_matmul: ctx is NULL");
  fp_status s = check_matmul(p, m, n, k, A, lda, B, ldb, C, ldc, algo);
  if (s != FP_OK) return s;
  return launch_matmul(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, algo, as_stream(stream));
}

extern "C" fp_status fp_matmul_grouped(fp_ctx ctx, const fp_mm_problem* problems, size_t count, int algo,
                                       void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_matmul_grouped: ctx is NULL");
  FP_CHECK(count == 0 || problems != nullptr, FP_EINVAL, "fp_matmul_grouped: problems is NULL");
  FP_CHECK(algo >= FP_MM_AUTO && algo <= FP_MM_SPLIT_F64, FP_EINVAL, "bad algo %d", algo);
  for (size_t i = 0; i < count; ++i) {
    const fp_mm_problem& x = problems[i];
    fp_status s = check_matmul(x.p, x.m, x.n, x.k, x.A, x.lda, x.B, x.ldb, x.C, x.ldc, algo);
    if (s == FP_OK) s = mm_bound_check(x.p, x.k, algo);
    if (s != FP_OK) return s;
  }
  cudaStream_t st = as_stream(stream);
  // which problems run grouped: the direct e4m3 kernel (AUTO, PLAIN_F8) or the 16-bit kernel
  // (RIGHT_TC packed, PLAIN_TC plain); the rest one by one through fp_matmul's path
  // (every problem passed mm_bound_check, so RIGHT_TC / PLAIN_TC problems all qualify)
  const bool f8 = algo == FP_MM_AUTO || algo == FP_MM_PLAIN_F8;
  const bool t16 = algo == FP_MM_RIGHT_TC || algo == FP_MM_PLAIN_TC;
  auto grouped = [&](const fp_mm_problem& x) {
    return (f8 && f8_direct_ok(x.p, x.k, x.A, x.lda, x.B, x.ldb)) || t16;
  };
  std::vector<const fp_mm_problem*> grp;
  for (size_t i = 0; i < count; ++i)
    if (grouped(problems[i])) grp.push_back(&problems[i]);
  if (!grp.empty()) {
    fp_status s = f8 ? launch_mm_f8_grouped(ctx, grp.data(), grp.size(), st)
                     : launch_mm_t16_grouped(ctx, grp.data(), grp.size(), algo == FP_MM_RIGHT_TC, st);
    if (s != FP_OK) return s;
  }
  for (size_t i = 0; i < count; ++i) {
    const fp_mm_problem& x = problems[i];
    if (grouped(x)) continue;
    fp_status s = launch_matmul(ctx, x.p, x.m, x.n, x.k, x.A, x.lda, x.B, x.ldb, x.C, x.ldc, algo, st);
    if (s != FP_OK) return s;
  }
  return FP_OK;
}

extern "C" fp_status fp_pack_cb(fp_ctx ctx, uint32_t p, int k, int n, const uint8_t* B, int ldb,
                                uint32_t b, uint32_t e, uint32_t word, void* CB, void* stream) {
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_pack_cb: ctx is NULL");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "p=%u not a prime <= 251", p);
  FP_CHECK(k >= 1 && n >= 1 && ldb >= n, FP_EINVAL, "fp_pack_cb: bad sizes");
  FP_CHECK(e >= 1 && e <= 16 && b >= 1 && b <= 32, FP_EINVAL, "fp_pack_cb: bad b/e");
  FP_CHECK(word == FP_WORD_F64 || word == FP_WORD_F32 || word == FP_WORD_U64, FP_EINVAL,
           "fp_pack_cb: word must be F64, F32 or U64");
  int beta = word_beta(word);
  unsigned __int128 tot = 0;
  for (uint32_t t = 0; t < e; ++t) {
    FP_CHECK((uint64_t)t * b < 100, FP_EBOUND, "fp_pack_cb: packed word exceeds the word");
    tot += ((unsigned __int128)(p - 1)) << (t * b);
  }
  FP_CHECK(tot < ((unsigned __int128)1 << (word == FP_WORD_F32 ? 24 : beta)), FP_EBOUND,
           "fp_pack_cb: e=%u residues at Q=2^%u exceed the word", e, b);
  FP_CHECK(B && CB, FP_EINVAL, "fp_pack_cb: null array");
  return launch_pack_cb(ctx, p, k, n, B, ldb, b, e, word, CB, as_stream(stream));
}
