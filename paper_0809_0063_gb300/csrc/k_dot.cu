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

// Grid-stride walk over the 16-byte vectors of u and v with four vector pairs loaded before any
// is used (128 bytes in flight per thread), as streaming loads that are evicted first: 2^28 pairs
// measured 0.77 / 0.82 of the HBM copy rate (packed / plain) against 0.70 / 0.71 with plain
// read-only loads, and eight pairs per thread ran slower (occupancy).  The vectors are visited
// in a different order than a plain stride loop; every consumer only sums exact integers.
template <typename Fn>
__device__ __forceinline__ void dot_vectors(const uint8_t* u, const uint8_t* v, uint64_t nv, Fn&& fn) {
  const uint4* U = reinterpret_cast<const uint4*>(u);
  const uint4* V = reinterpret_cast<const uint4*>(v);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < nv; i += 4 * stride) {
    uint4 a[4], c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = __ldcs(U + i + j * stride);     // streaming: read once, evict first
      c[j] = __ldcs(V + i + j * stride);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) fn(a[j], c[j]);
  }
  for (; i < nv; i += stride) fn(__ldcs(U + i), __ldcs(V + i));
}

__global__ void __launch_bounds__(256) k_dot_plain(const uint8_t* __restrict__ u, const uint8_t* __restrict__ v,
                                                   uint64_t n, uint64_t* __restrict__ partial, uint32_t p,
                                                   uint32_t* err) {
  uint64_t acc = 0;
  uint32_t bad = 0;
  bool aligned = ((((uintptr_t)u) | ((uintptr_t)v)) & 15u) == 0;
  uint64_t nv = aligned ? n / 16 : 0;
  const uint32_t pp = 0x01010101u * p;
  dot_vectors(u, v, nv, [&](const uint4& a, const uint4& b) {
    uint32_t s = 0;
    s = __dp4a(a.x, b.x, s);
    s = __dp4a(a.y, b.y, s);
    s = __dp4a(a.z, b.z, s);
    s = __dp4a(a.w, b.w, s);
    acc += s;
    // range check: some byte >= p
    bad |= __vcmpgeu4(a.x, pp) | __vcmpgeu4(a.y, pp) | __vcmpgeu4(a.z, pp) | __vcmpgeu4(a.w, pp);
    bad |= __vcmpgeu4(b.x, pp) | __vcmpgeu4(b.y, pp) | __vcmpgeu4(b.z, pp) | __vcmpgeu4(b.w, pp);
  });
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

// The same middle product on 16-byte vectors: each thread takes 16 entries of u and of v at a
// time (16 / D1 blocks of D1 entries, D1 in {2, 4, 8}), packs every block reversed (u) and
// forward (v) at Q = 2^b from the bytes in registers, and accumulates the u64 word products;
// every F blocks the digit of Q^(D1-1) -- the block dot products summed -- is moved out to a
// u64 sum.  Range check on whole words.  The < 16 entries past the last full vector are added
// plainly by thread 0 of block 0.
template <int D1>
__global__ void __launch_bounds__(256) k_dot_dqt_vec(const uint8_t* __restrict__ u, const uint8_t* __restrict__ v,
                                                     uint64_t n, uint64_t* __restrict__ partial, uint32_t p,
                                                     uint32_t b, uint32_t F, uint32_t* err) {
  constexpr int BPV = 16 / D1;                         // blocks per vector
  const uint64_t nv = n / 16;
  const uint64_t mask = (1ull << b) - 1;
  const uint32_t mid = (D1 - 1) * b;
  const uint32_t pp = 0x01010101u * p;
  uint64_t sum = 0, acc = 0;
  uint32_t cnt = 0, bad = 0;
  dot_vectors(u, v, nv, [&](const uint4& a, const uint4& c) {
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) bad |= __vcmpgeu4(wa[q], pp) | __vcmpgeu4(wc[q], pp);
    if (cnt + BPV > F) {                               // the next BPV blocks would overflow a digit
      sum += (acc >> mid) & mask;
      acc = 0;
      cnt = 0;
    }
#pragma unroll
    for (int j = 0; j < BPV; ++j) {
      uint64_t wl = 0, wr = 0;
#pragma unroll
      for (int t = 0; t < D1; ++t) {
        const int e = j * D1 + t;                      // entry within the vector
        const uint64_t ea = (wa[e >> 2] >> (8 * (e & 3))) & 0xffu, ec = (wc[e >> 2] >> (8 * (e & 3))) & 0xffu;
        wl |= ea << ((D1 - 1 - t) * b);                // reversed: entry t gets Q^(D1-1-t)
        wr |= ec << (t * b);                           // forward
      }
      acc += wl * wr;
    }
    cnt += BPV;
  });
  sum += (acc >> mid) & mask;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (uint64_t i = nv * 16; i < n; ++i) {
      const uint32_t x = u[i], y = v[i];
      bad |= (x >= p) | (y >= p);
      sum += x * y;
    }
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

// The middle product at a byte-aligned Q, where packing is a byte permutation of the loaded
// words.  QB = 8: blocks of 4 entries (one 32-bit word), Q = 2^8: the forward word of v is the
// little-endian word as loaded, the reversed word of u is its byte reversal, and the digit of
// Q^3 of their product is the block dot product (p <= 7).  QB = 16: blocks of 2 entries, each
// spread to 16-bit fields by one permutation (p <= 181).  One 32 x 32 -> 64-bit multiply-add per
// block; every F blocks the middle digit is moved out.  Tail entries as in k_dot_dqt_vec.
template <int QB>
__global__ void __launch_bounds__(256) k_dot_dqt_bytes(const uint8_t* __restrict__ u, const uint8_t* __restrict__ v,
                                                       uint64_t n, uint64_t* __restrict__ partial, uint32_t p,
                                                       uint32_t F, uint32_t* err) {
  const uint64_t nv = n / 16;
  constexpr uint32_t MID = QB == 8 ? 24 : 16;
  constexpr uint64_t MASK = QB == 8 ? 0xffull : 0xffffull;
  const uint32_t pp = 0x01010101u * p;
  uint64_t sum = 0, acc = 0;
  uint32_t cnt = 0, bad = 0;
  dot_vectors(u, v, nv, [&](const uint4& a, const uint4& c) {
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bad |= __vcmpgeu4(wa[q], pp) | __vcmpgeu4(wc[q], pp);
      if (QB == 8) {
        if (cnt == F) {
          sum += (acc >> MID) & MASK;
          acc = 0;
          cnt = 0;
        }
        acc += (uint64_t)__byte_perm(wa[q], 0, 0x0123) * wc[q];
        ++cnt;
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (cnt == F) {
            sum += (acc >> MID) & MASK;
            acc = 0;
            cnt = 0;
          }
          // entries 2h, 2h+1: u reversed (u_2h at Q), v forward (v_2h at 1), 16-bit fields
          const uint32_t wl = __byte_perm(wa[q], 0, h ? 0x4243u : 0x4041u);
          const uint32_t wr = __byte_perm(wc[q], 0, h ? 0x4342u : 0x4140u);
          acc += (uint64_t)wl * wr;
          ++cnt;
        }
      }
    }
  });
  sum += (acc >> MID) & MASK;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (uint64_t i = nv * 16; i < n; ++i) {
      const uint32_t x = u[i], y = v[i];
      bad |= (x >= p) | (y >= p);
      sum += x * y;
    }
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

// Parameters for the vector kernel: the largest D1 in {8, 4, 2} with at least one vector's
// 16 / D1 blocks per accumulation (F >= 16 / D1) and the 2 D1 - 1 digits within 64 bits.
static bool dot_dqt_vec_params(uint32_t p, uint32_t& D1, uint32_t& b, uint32_t& F) {
  uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  if (pp == 0) pp = 1;
  for (uint32_t d1 = 8; d1 >= 2; d1 /= 2) {
    uint32_t bb = 64 / (2 * d1 - 1);
    if (bb > 32) bb = 32;
    const uint64_t f = ((1ull << bb) - 1) / (d1 * pp);
    if (f >= 16 / d1) {
      D1 = d1;
      b = bb;
      F = (uint32_t)(f > 1024 ? 1024 : f);
      return true;
    }
  }
  return false;
}

// The packed stream: the vector kernel when both arrays are 16-byte aligned and a vector
// packing fits, else the entry-by-entry kernel.
static void dot_dqt_launch(const uint8_t* u, const uint8_t* v, size_t n, uint64_t* partial, uint32_t p, uint32_t D1,
                           uint32_t b, uint32_t F, int grid, cudaStream_t st, uint32_t* err) {
  uint32_t vD1, vb, vF;
  const bool aligned = ((((uintptr_t)u) | ((uintptr_t)v)) & 15u) == 0;
  const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
  // byte-aligned Q: F blocks with F D1 (p-1)^2 < Q (every digit of the accumulated word)
  if (aligned && p <= 7 && 4 * pp < 256) {
    k_dot_dqt_bytes<8><<<grid, 256, 0, st>>>(u, v, n, partial, p, (uint32_t)(255 / (4 * (pp ? pp : 1))), err);
  } else if (aligned && 2 * pp < 65536) {
    const uint64_t f = 65535 / (2 * (pp ? pp : 1));
    k_dot_dqt_bytes<16><<<grid, 256, 0, st>>>(u, v, n, partial, p, (uint32_t)(f > 4096 ? 4096 : f), err);
  } else if (aligned && dot_dqt_vec_params(p, vD1, vb, vF)) {
    if (vD1 == 8) k_dot_dqt_vec<8><<<grid, 256, 0, st>>>(u, v, n, partial, p, vb, vF, err);
    else if (vD1 == 4) k_dot_dqt_vec<4><<<grid, 256, 0, st>>>(u, v, n, partial, p, vb, vF, err);
    else k_dot_dqt_vec<2><<<grid, 256, 0, st>>>(u, v, n, partial, p, vb, vF, err);
  } else {
    k_dot_dqt<<<grid, 256, 0, st>>>(u, v, n, partial, p, D1, b, F, err);
  }
}

fp_status launch_dot(fp_ctx ctx, uint32_t p, const uint8_t* u, const uint8_t* v, size_t n, uint32_t* out,
                     int algo, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  int grid = ctx->num_sms * 4;
  fp_status s = ensure_scratch(ctx, (size_t)grid * sizeof(uint64_t), 1, st);
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
    FP_LAUNCH(ctx, "k_dot_dqt", st, dot_dqt_launch(u, v, n, partial, p, D1, b, F, grid, st, ctx->d_err));
  } else if (algo == FP_ALGO_AUTO && dqt) {
    // both are HBM streams; the packed one issues fewer multiplies per byte only for small p,
    // the plain dp4a stream is the cheaper instruction mix: AUTO takes the packed route
    // (the method) when it packs at least 4 entries per word.
    if (D1 >= 4) FP_LAUNCH(ctx, "k_dot_dqt", st, dot_dqt_launch(u, v, n, partial, p, D1, b, F, grid, st, ctx->d_err));
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
    dot_dqt_launch(u, v, n, partial, p, D1, b, F, grid, st, err);
  else
    k_dot_plain<<<grid, 256, 0, st>>>(u, v, n, partial, p, err);
  FP_CUDA(cudaGetLastError());
  k_dot_final_noalloc<<<1, 1024, 0, st>>>(partial, grid, out, p, err);
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}
