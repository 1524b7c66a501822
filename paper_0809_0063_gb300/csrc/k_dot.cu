// Modular dot product (Algorithm 1 with degree-0 entries).
//  plain : dp4a on 16-byte vectors, per-thread u64 sums (delayed reduction, Eq. delayed), one
//          reduction mod p at the very end.
//  DQT   : middle product of Sec. 7.1: blocks of d+1 entries packed reversed on the left,
//          forward on the right, one u64 word product per block; the coefficient of Q^d of the
//          accumulated words is the block dot product; F blocks are accumulated per word with
//          F (d+1)(p-1)^2 < Q so no digit carries, then the middle digit is extracted.
// Both are HBM-bound streams; per-block u64 partial sums go to context scratch and one
// final block reduces them and applies the single mod p.
#include "fpdqt_internal.cuh"

namespace fpd {

__global__ void __launch_bounds__(256) k_dot_plain(const uint8_t* __restrict__ u, const uint8_t* __restrict__ v,
                                                   uint64_t n, uint64_t* __restrict__ partial, uint32_t p,
                                                   uint32_t* err) {
  uint64_t acc = 0;
  uint32_t bad = 0;
  bool aligned = ((((uintptr_t)u) | ((uintptr_t)v)) & 15u) == 0;
  uint64_t nv = aligned ? n / 16 : 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 a = __ldg(reinterpret_cast<const uint4*>(u) + i);
    uint4 b = __ldg(reinterpret_cast<const uint4*>(v) + i);
    uint32_t s = 0;
    s = __dp4a(a.x, b.x, s);
    s = __dp4a(a.y, b.y, s);
    s = __dp4a(a.z, b.z, s);
    s = __dp4a(a.w, b.w, s);
    acc += s;
    // range check: a byte >= p exists iff max byte >= p; use __vcmpgeu4
    uint32_t pp = 0x01010101u * p;
    bad |= __vcmpgeu4(a.x, pp) | __vcmpgeu4(a.y, pp) | __vcmpgeu4(a.z, pp) | __vcmpgeu4(a.w, pp);
    bad |= __vcmpgeu4(b.x, pp) | __vcmpgeu4(b.y, pp) | __vcmpgeu4(b.z, pp) | __vcmpgeu4(b.w, pp);
  }
  for (uint64_t i = nv * 16 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t a = u[i], b = v[i];
    bad |= (a >= p) | (b >= p);
    acc += a * b;
  }
  // block reduction
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ uint64_t ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// Middle-product DQT dot, d+1 = D1 entries per word at Q = 2^b; F blocks per accumulation.
__global__ void __launch_bounds__(256) k_dot_dqt(const uint8_t* __restrict__ u, const uint8_t* __restrict__ v,
                                                 uint64_t n, uint64_t* __restrict__ partial, uint32_t p,
                                                 uint32_t D1, uint32_t b, uint32_t F, uint32_t* err) {
  const uint64_t nblk = (n + D1 - 1) / D1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t mask = (1ull << b) - 1;
  const uint32_t mid = (D1 - 1) * b;
  uint64_t sum = 0, acc = 0;
  uint32_t cnt = 0, bad = 0;
  for (uint64_t blk = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; blk < nblk; blk += stride) {
    uint64_t wl = 0, wr = 0;
    const uint64_t base = blk * D1;
    for (uint32_t t = 0; t < D1; ++t) {
      uint64_t idx = base + t;
      uint32_t a = idx < n ? u[idx] : 0u, c = idx < n ? v[idx] : 0u;
      bad |= (a >= p) | (c >= p);
      wl = (wl << b) | a;                  // reversed: u_{base} gets Q^{d}
      wr |= (uint64_t)c << (t * b);        // forward:  v_{base+t} gets Q^t
    }
    acc += wl * wr;
    if (++cnt == F) {
      sum += (acc >> mid) & mask;
      acc = 0;
      cnt = 0;
    }
  }
  sum += (acc >> mid) & mask;
  for (int o = 16; o; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  __shared__ uint64_t ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
  if (bad) flag_error(err, ERR_RANGE);
}

__global__ void k_dot_final(const uint64_t* __restrict__ partial, int nparts, uint32_t* out, uint32_t p) {
  uint64_t t = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += partial[i] % p;
  for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  __shared__ uint64_t ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    *out = (uint32_t)(s % p);
  }
}

// Middle-product parameters: largest D1 <= 8 with Q = 2^b > F D1 (p-1)^2 for some F >= 1 and
// the accumulated word (2 D1 - 1 digits of at most F D1 (p-1)^2) below 2^64; F as large as
// the word allows.
static bool dot_dqt_params(uint32_t p, uint32_t& D1, uint32_t& b, uint32_t& F) {
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  if (pp == 0) pp = 1;
  for (uint32_t d1 = 8; d1 >= 2; --d1) {
    uint32_t nd = 2 * d1 - 1;
    uint32_t bb = 64 / nd;  // digits of bb bits; the sum of digit bounds < 2^64 when each < 2^bb
    if (bb > 32) bb = 32;
    uint64_t Q = 1ull << bb;
    uint64_t f = (Q - 1) / (d1 * pp);
    if (f >= 1) {
      D1 = d1;
      b = bb;
      F = (uint32_t)(f > 1024 ? 1024 : f);
      return true;
    }
  }
  return false;
}

fp_status launch_dot(fp_ctx ctx, uint32_t p, const uint8_t* u, const uint8_t* v, size_t n, uint32_t* out,
                     int algo, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  int grid = ctx->num_sms * 4;
  fp_status s = ensure_scratch(ctx, (size_t)grid * sizeof(uint64_t), 1);
  if (s != FP_OK) return s;
  uint64_t* partial = (uint64_t*)ctx->scratch2;
  if (n == 0) {
    FP_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), st));
    return FP_OK;
  }
  uint32_t D1 = 0, b = 0, F = 0;
  bool dqt = algo != FP_ALGO_PLAIN && dot_dqt_params(p, D1, b, F);
  if (algo != FP_ALGO_PLAIN && algo != FP_ALGO_AUTO && !dqt) {
    set_error("fp_dot: no middle-product packing fits for p=%u", p);
    return FP_EBOUND;
  }
  if (dqt && algo != FP_ALGO_AUTO) {
    FP_LAUNCH(ctx, "k_dot_dqt", st, k_dot_dqt<<<grid, 256, 0, st>>>(u, v, n, partial, p, D1, b, F, ctx->d_err));
  } else if (algo == FP_ALGO_AUTO && dqt) {
    // both are HBM streams; the packed one issues fewer multiplies per byte only for small p,
    // the plain dp4a stream is the cheaper instruction mix: AUTO takes the packed route
    // (the method) when it packs at least 4 entries per word.
    if (D1 >= 4) FP_LAUNCH(ctx, "k_dot_dqt", st, k_dot_dqt<<<grid, 256, 0, st>>>(u, v, n, partial, p, D1, b, F, ctx->d_err));
    else FP_LAUNCH(ctx, "k_dot_plain", st, k_dot_plain<<<grid, 256, 0, st>>>(u, v, n, partial, p, ctx->d_err));
  } else {
    FP_LAUNCH(ctx, "k_dot_plain", st, k_dot_plain<<<grid, 256, 0, st>>>(u, v, n, partial, p, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  FP_LAUNCH(ctx, "k_dot_final", st, k_dot_final<<<1, 1024, 0, st>>>(partial, grid, out, p));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

// ------------------------------------------------------------------ allocation-free variant
//
// For callers that cannot allocate device memory.  The scratch is this file-scope array in the
// device image: FP_DOT_NOALLOC_MAX_PARTIALS 64-bit partial sums followed by one 32-bit error
// word.  Partials are always written before they are read, so only the error word is cleared
// at the start of each call.

static __device__ __align__(256) uint64_t g_dot_noalloc_scratch[FP_DOT_NOALLOC_MAX_PARTIALS + 32];

// The name above is a host-side stand-in in host code; the device address is looked up once
// per device (with that device current) and cached here.
static constexpr int NOALLOC_MAX_DEVICES = 64;
static uint64_t* g_dot_noalloc_ptr[NOALLOC_MAX_DEVICES];
static int g_dot_noalloc_sms[NOALLOC_MAX_DEVICES];
static std::mutex g_dot_noalloc_mu;

static fp_status dot_noalloc_setup(int dev, uint64_t** ptr, int* sms) {
  std::lock_guard<std::mutex> lk(g_dot_noalloc_mu);
  if (!g_dot_noalloc_ptr[dev]) {
    uint64_t* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_dot_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fp_dot_noalloc scratch)");
    int n_sms = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_dot_noalloc_sms[dev] = n_sms;
    g_dot_noalloc_ptr[dev] = p;
  }
  *ptr = g_dot_noalloc_ptr[dev];
  *sms = g_dot_noalloc_sms[dev];
  return FP_OK;
}

__global__ void k_dot_final_noalloc(const uint64_t* __restrict__ partial, int nparts, uint32_t* out, uint32_t p,
                                    const uint32_t* err) {
  uint64_t t = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += partial[i] % p;
  for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  __shared__ uint64_t ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    *out = *err ? 0xFFFFFFFFu : (uint32_t)(s % p);
  }
}

}  // namespace fpd

extern "C" fp_status fp_dot_noalloc(uint32_t p, const uint8_t* u, const uint8_t* v, size_t n, uint32_t* out,
                                    int algo, void* stream) {
  using namespace fpd;
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "fp_dot_noalloc: p=%u not a prime <= 251", p);
  FP_CHECK(out != nullptr, FP_EINVAL, "fp_dot_noalloc: out is NULL");
  FP_CHECK(n <= (1ull << 40), FP_EINVAL, "fp_dot_noalloc: n=%zu above the 2^40 limit", n);
  FP_CHECK(algo >= FP_ALGO_AUTO && algo <= FP_ALGO_DQT_U32, FP_EINVAL, "fp_dot_noalloc: bad algo %d", algo);
  FP_CHECK(n == 0 || (u && v), FP_EINVAL, "fp_dot_noalloc: null array");
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  FP_CHECK(dev >= 0 && dev < NOALLOC_MAX_DEVICES, FP_EUNSUPPORTED, "fp_dot_noalloc: device %d", dev);
  uint64_t* scratch = nullptr;
  int sms = 0;
  fp_status s = dot_noalloc_setup(dev, &scratch, &sms);
  if (s != FP_OK) return s;
  const int grid = sms * 4;
  FP_CHECK(grid >= 1 && grid <= FP_DOT_NOALLOC_MAX_PARTIALS, FP_EUNSUPPORTED,
           "fp_dot_noalloc: %d partial sums needed, the fixed scratch holds %d", grid, FP_DOT_NOALLOC_MAX_PARTIALS);
  cudaStream_t st = as_stream(stream);
  if (n == 0) {
    FP_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), st));
    return FP_OK;
  }
  uint64_t* partial = scratch;
  uint32_t* err = reinterpret_cast<uint32_t*>(scratch + FP_DOT_NOALLOC_MAX_PARTIALS);
  FP_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
  uint32_t D1 = 0, b = 0, F = 0;
  bool dqt = algo != FP_ALGO_PLAIN && dot_dqt_params(p, D1, b, F);
  if (algo != FP_ALGO_PLAIN && algo != FP_ALGO_AUTO && !dqt) {
    set_error("fp_dot_noalloc: no middle-product packing fits for p=%u", p);
    return FP_EBOUND;
  }
  if (dqt && (algo != FP_ALGO_AUTO || D1 >= 4))
    k_dot_dqt<<<grid, 256, 0, st>>>(u, v, n, partial, p, D1, b, F, err);
  else
    k_dot_plain<<<grid, 256, 0, st>>>(u, v, n, partial, p, err);
  FP_CUDA(cudaGetLastError());
  k_dot_final_noalloc<<<1, 1024, 0, st>>>(partial, grid, out, p, err);
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}
