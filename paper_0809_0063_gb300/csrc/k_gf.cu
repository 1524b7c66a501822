// GF(p^k) multiplication by Algorithm FGDP (Sec. 6) with n = 1, on the device:
//   1. table DQT: element index -> u64 word sum_i c_i q^i (one shared-memory lookup),
//   2. one word product,
//   3. REDQ COMPRESSION: u_i = floor(r/q^i) - p floor(s/q^i), i = 0..2k-2 (no correction),
//   4./5. L[u_0..u_{k-1}] and H[u_{k-1}..u_{2k-2}] (Theorem fgdp), each already reduced modulo
//      the field's modulus, indexed in the binary format sum u_i 2^{c i}, c = ceil(log2 p)
//      (Note on Indexing),
//   6. one field addition.
// L and H entries hold the coefficient vector "spread" in 4-bit fields (p <= 7) or 8-bit fields,
// so the field addition is one integer add and a per-field conditional subtraction of p.
#include <algorithm>
#include <vector>

#include "fpdqt_internal.cuh"
#include "stream.cuh"

struct fp_gf_s {
  uint32_t p = 0, k = 0, b = 0, c = 0, fb = 0;  // q = 2^b; index bits per residue c; field bits fb
  uint32_t order = 0;                            // p^k
  uint32_t elem_bytes = 1;
  std::vector<uint32_t> modulus;                 // k+1 coefficients, constant first, monic
  uint64_t* d_word = nullptr;                    // [p^k]
  uint32_t* d_L = nullptr;                       // [2^{c k}]
  uint32_t* d_H = nullptr;                       // [2^{c k}]
  fpd::RedqParams P{};
  int device = 0;
};

namespace fpd {

// ---------------------------------------------------------------- host field construction

static std::vector<uint32_t> poly_rem(std::vector<uint32_t> a, const std::vector<uint32_t>& m, uint32_t p) {
  int k = (int)m.size() - 1;
  for (int d = (int)a.size() - 1; d >= k; --d) {
    uint32_t lead = a[d] % p;
    if (!lead) continue;
    for (int i = 0; i <= k; ++i) a[d - k + i] = (a[d - k + i] + (p - lead) * m[i]) % p;
  }
  a.resize(k);
  return a;
}

static bool irreducible(const std::vector<uint32_t>& f, uint32_t p) {
  int k = (int)f.size() - 1;
  for (int deg = 1; deg <= k / 2; ++deg) {
    uint64_t cnt = 1;
    for (int i = 0; i < deg; ++i) cnt *= p;
    for (uint64_t key = 0; key < cnt; ++key) {
      std::vector<uint32_t> g(deg + 1);
      uint64_t x = key;
      for (int i = 0; i < deg; ++i) { g[i] = (uint32_t)(x % p); x /= p; }
      g[deg] = 1;
      std::vector<uint32_t> r = poly_rem(f, g, p);
      bool zero = true;
      for (uint32_t v : r) zero &= v == 0;
      if (zero) return false;
    }
  }
  return true;
}

static uint32_t spread(const std::vector<uint32_t>& coeffs, uint32_t fb) {
  uint32_t s = 0;
  for (size_t i = 0; i < coeffs.size(); ++i) s |= coeffs[i] << (i * fb);
  return s;
}

// ---------------------------------------------------------------- kernel

struct GfDev {
  const uint64_t* word;
  const uint32_t* L;
  const uint32_t* H;
  uint32_t order, k, cbits, fb;
  uint32_t ones;   // one bit at the bottom of each of the k fields of fb bits
};

// Shared copies of the three tables (word table, L, H) for one block.
__device__ __forceinline__ void gf_load_tables(const GfDev& G, uint8_t* sm, uint64_t*& sw, uint32_t*& sL,
                                               uint32_t*& sH) {
  sw = reinterpret_cast<uint64_t*>(sm);
  const uint32_t tsz = 1u << (G.cbits * G.k);
  sL = reinterpret_cast<uint32_t*>(sw + G.order);
  sH = sL + tsz;
  for (uint32_t i = threadIdx.x; i < G.order; i += blockDim.x) sw[i] = G.word[i];
  for (uint32_t i = threadIdx.x; i < tsz; i += blockDim.x) { sL[i] = G.L[i]; sH[i] = G.H[i]; }
  __syncthreads();
}

// One product by Algorithm FGDP with n = 1 (see the file comment).
__device__ __forceinline__ uint32_t gf_mul_one(uint32_t xa, uint32_t xb, const GfDev& G, const uint64_t* sw,
                                               const uint32_t* sL, const uint32_t* sH, const RedqParams& P,
                                               uint32_t& bad) {
  const uint32_t p = P.p, bq = P.b, k = G.k, fb = G.fb, cbits = G.cbits;
  bad |= (xa >= G.order) | (xb >= G.order);
  xa = xa < G.order ? xa : 0u;
  xb = xb < G.order ? xb : 0u;
  const uint64_t r = sw[xa] * sw[xb];             // lines 1-2
  const uint64_t s = divp64(r, P.dv);             // REDQ compression quotient (line 3)
  const uint32_t rl = (uint32_t)r, rh = (uint32_t)(r >> 32);
  const uint32_t sl = (uint32_t)s, shh = (uint32_t)(s >> 32);
  const uint32_t qmask = (1u << bq) - 1u;
  uint32_t il = 0, ih = 0;
  for (uint32_t j = 0, sh = 0; j < 2 * k - 1; ++j, sh += bq) {
    // low 32 bits of r >> sh and s >> sh by funnel shifts (only the low bq bits matter)
    const uint32_t rr = sh < 32 ? __funnelshift_r(rl, rh, sh) : (rh >> (sh - 32));
    const uint32_t ss = sh < 32 ? __funnelshift_r(sl, shh, sh) : (shh >> (sh - 32));
    const uint32_t uj = (rr - p * ss) & qmask;
    if (j < k) il |= uj << (j * cbits);
    if (j + 1 >= k) ih |= uj << ((j + 1 - k) * cbits);
  }
  const uint32_t hb = fb - 1;                     // bit tested after adding 2^hb - p per field
  uint32_t x = sL[il] + sH[ih];                    // lines 4-6: two lookups, one field add
  const uint32_t ge = ((x + ((1u << hb) - p) * G.ones) >> hb) & G.ones;
  x -= p * ge;
  const uint32_t fmask = (1u << fb) - 1u;
  uint32_t idx = 0;
  for (int j = (int)k - 1; j >= 0; --j) idx = idx * p + ((x >> (j * fb)) & fmask);
  return idx;
}

template <typename E>
__global__ void __launch_bounds__(256) k_gf_mul(const E* __restrict__ a, const E* __restrict__ b, E* __restrict__ c,
                                                uint64_t count, GfDev G, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(G, sm, sw, sL, sH);
  uint32_t bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + stride < count; i += 2 * stride) {   // two independent products per trip (ILP)
    const uint32_t x0 = a[i], y0 = b[i], x1 = a[i + stride], y1 = b[i + stride];
    const uint32_t r0 = gf_mul_one(x0, y0, G, sw, sL, sH, P, bad);
    const uint32_t r1 = gf_mul_one(x1, y1, G, sw, sL, sH, P, bad);
    c[i] = (E)r0;
    c[i + stride] = (E)r1;
  }
  if (i < count) c[i] = (E)gf_mul_one(a[i], b[i], G, sw, sL, sH, P, bad);
  if (bad) flag_error(err, ERR_RANGE);
}

// The batched multiply on the bulk-copy streaming loop: 4096 pairs per tile.
template <typename E>
struct GfOp {
  static constexpr uint32_t IPT = 16;
  static constexpr uint32_t UNROLL = 4;
  GfDev G;
  RedqParams P;
  const uint64_t* sw;
  const uint32_t *sL, *sH;
  uint32_t bad;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t* b, uint8_t* out) {
    *reinterpret_cast<E*>(out) = (E)gf_mul_one(*reinterpret_cast<const E*>(a), *reinterpret_cast<const E*>(b), G, sw,
                                               sL, sH, P, bad);
  }
};

template <typename E>
__global__ void __launch_bounds__(256) k_gf_mul_bulk(const E* __restrict__ a, const E* __restrict__ b, E* __restrict__ c,
                                                     uint64_t ntiles, uint32_t table_bytes, GfDev G, RedqParams P,
                                                     uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(G, sm, sw, sL, sH);
  GfOp<E> op{G, P, sw, sL, sH, 0};
  stream_tiles(op, reinterpret_cast<const uint8_t*>(a), reinterpret_cast<const uint8_t*>(b),
               reinterpret_cast<uint8_t*>(c), ntiles, sizeof(E), sizeof(E), sizeof(E), sm + table_bytes, err);
  if (op.bad) flag_error(err, ERR_RANGE);
}

// ------------------------------------------------------------------ compile-time fields

// The parameters fp_gf_create chooses for GF(P^K), as compile-time constants (same rules).
template <uint32_t P, uint32_t K>
struct GfConst {
  static constexpr uint32_t order() { uint32_t o = 1; for (uint32_t i = 0; i < K; ++i) o *= P; return o; }
  static constexpr uint32_t cbits() { uint32_t c = 0; while ((1u << c) < P) ++c; return c; }
  static constexpr uint32_t fbits() {
    uint32_t f = 1;
    while ((1u << (f - 1)) < P || (1u << f) <= 2 * P - 2 + (1u << (f - 1)) - P) ++f;
    return f;
  }
  static constexpr uint32_t qbits() {
    uint32_t b = 1;
    while ((1ull << b) <= (uint64_t)K * (P - 1) * (P - 1) || (1ull << b) < P) ++b;
    return b;
  }
  static constexpr uint32_t ORDER = order(), CB = cbits(), FB = fbits(), B = qbits();
  static constexpr uint32_t ONES = [] { uint32_t o = 0; for (uint32_t i = 0; i < K; ++i) o |= 1u << (i * FB); return o; }();
};

// One product by Algorithm FGDP (n = 1) with every shift, mask and loop bound fixed at
// compile time: the same steps as gf_mul_one.
template <uint32_t P, uint32_t K>
__device__ __forceinline__ uint32_t gf_mul_fixed(uint32_t xa, uint32_t xb, const uint64_t* sw, const uint32_t* sL,
                                                 const uint32_t* sH, uint32_t& bad) {
  using F = GfConst<P, K>;
  bad |= (xa >= F::ORDER) | (xb >= F::ORDER);
  xa = xa < F::ORDER ? xa : 0u;
  xb = xb < F::ORDER ? xb : 0u;
  const uint64_t r = sw[xa] * sw[xb];             // table DQT of both operands, one word product
  const uint64_t s = r / P;                       // REDQ compression quotient
  uint32_t il = 0, ih = 0;
#pragma unroll
  for (uint32_t j = 0; j < 2 * K - 1; ++j) {
    const uint32_t uj = ((uint32_t)(r >> (j * F::B)) - P * (uint32_t)(s >> (j * F::B))) & ((1u << F::B) - 1u);
    if (j < K) il |= uj << (j * F::CB);
    if (j + 1 >= K) ih |= uj << ((j + 1 - K) * F::CB);
  }
  constexpr uint32_t HB = F::FB - 1;
  uint32_t x = sL[il] + sH[ih];                    // two lookups, one field addition
  const uint32_t ge = ((x + ((1u << HB) - P) * F::ONES) >> HB) & F::ONES;
  x -= P * ge;
  uint32_t idx = 0;
#pragma unroll
  for (int j = (int)K - 1; j >= 0; --j) idx = idx * P + ((x >> (j * F::FB)) & ((1u << F::FB) - 1u));
  return idx;
}

// Four products per item, so that every shared-memory access of the stream is a whole
// 32-bit word (uint8 elements) or a pair of words (uint16).
template <uint32_t P, uint32_t K, typename E>
struct GfFixedOp {
  static constexpr uint32_t IPT = 4;
  static constexpr uint32_t UNROLL = 2;
  const uint64_t* sw;
  const uint32_t *sL, *sH;
  uint32_t bad;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t* b, uint8_t* out) {
    if (sizeof(E) == 1) {
      const uint32_t wa = *reinterpret_cast<const uint32_t*>(a), wb = *reinterpret_cast<const uint32_t*>(b);
      uint32_t wc = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        wc |= gf_mul_fixed<P, K>((wa >> (8 * j)) & 0xffu, (wb >> (8 * j)) & 0xffu, sw, sL, sH, bad) << (8 * j);
      *reinterpret_cast<uint32_t*>(out) = wc;
    } else {
      const uint2 wa = *reinterpret_cast<const uint2*>(a), wb = *reinterpret_cast<const uint2*>(b);
      const uint32_t c0 = gf_mul_fixed<P, K>(wa.x & 0xffffu, wb.x & 0xffffu, sw, sL, sH, bad);
      const uint32_t c1 = gf_mul_fixed<P, K>(wa.x >> 16, wb.x >> 16, sw, sL, sH, bad);
      const uint32_t c2 = gf_mul_fixed<P, K>(wa.y & 0xffffu, wb.y & 0xffffu, sw, sL, sH, bad);
      const uint32_t c3 = gf_mul_fixed<P, K>(wa.y >> 16, wb.y >> 16, sw, sL, sH, bad);
      *reinterpret_cast<uint2*>(out) = make_uint2(c0 | (c1 << 16), c2 | (c3 << 16));
    }
  }
};

template <uint32_t P, uint32_t K, typename E>
__global__ void __launch_bounds__(256) k_gf_mul_fixed(const E* __restrict__ a, const E* __restrict__ b,
                                                      E* __restrict__ c, uint64_t ntiles, uint32_t table_bytes,
                                                      GfDev G, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(G, sm, sw, sL, sH);
  GfFixedOp<P, K, E> op{sw, sL, sH, 0};
  stream_tiles(op, reinterpret_cast<const uint8_t*>(a), reinterpret_cast<const uint8_t*>(b),
               reinterpret_cast<uint8_t*>(c), ntiles, 4 * sizeof(E), 4 * sizeof(E), 4 * sizeof(E), sm + table_bytes,
               err);
  if (op.bad) flag_error(err, ERR_RANGE);
}

// Segmented form for the serving loop: segment s multiplies count[s] pairs at byte offsets
// a/b/c from `base`; one block per segment.
struct GfSeg { uint64_t a, b, c; uint32_t count, pad; };

template <typename E>
__global__ void __launch_bounds__(256) k_gf_mul_seg(uint8_t* base, const GfSeg* __restrict__ segs, uint32_t nseg,
                                                    GfDev G, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(G, sm, sw, sL, sH);
  uint32_t bad = 0;
  for (uint32_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const GfSeg S = segs[sg];
    const E* a = reinterpret_cast<const E*>(base + S.a);
    const E* b = reinterpret_cast<const E*>(base + S.b);
    E* c = reinterpret_cast<E*>(base + S.c);
    for (uint32_t i = threadIdx.x; i < S.count; i += blockDim.x) c[i] = (E)gf_mul_one(a[i], b[i], G, sw, sL, sH, P, bad);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

}  // namespace fpd

using namespace fpd;

extern "C" fp_status fp_gf_create(fp_ctx ctx, uint32_t p, uint32_t k, fp_gf* out) {
  FP_CHECK(ctx && out, FP_EINVAL, "fp_gf_create: null argument");
  *out = nullptr;
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "fp_gf_create: p=%u not a prime <= 251", p);
  FP_CHECK(k >= 1 && k <= 16, FP_EINVAL, "fp_gf_create: k=%u outside [1, 16]", k);
  uint64_t order = 1;
  for (uint32_t i = 0; i < k; ++i) order *= p;
  FP_CHECK(order <= 65536, FP_EINVAL, "fp_gf_create: p^k = %llu > 65536", (unsigned long long)order);
  uint32_t cbits = 0;
  while ((1u << cbits) < p) ++cbits;
  FP_CHECK(cbits * k <= 12, FP_EUNSUPPORTED,
           "fp_gf_create: binary-indexed L/H tables would need 2^%u entries", cbits * k);
  // field bits: each field must hold 2p-2 plus headroom for the compare trick (2^(fb-1) >= p)
  uint32_t fb = 1;
  while ((1u << (fb - 1)) < p || (1u << fb) <= 2 * p - 2 + (1u << (fb - 1)) - p) ++fb;
  FP_CHECK(fb * k <= 32, FP_EUNSUPPORTED, "fp_gf_create: spread form needs %u bits", fb * k);
  // q: smallest 2^b above the largest digit k (p-1)^2 of a product of two field elements
  uint64_t D = (uint64_t)k * (p - 1) * (p - 1);
  uint32_t b = 1;
  while ((1ull << b) <= D || (1ull << b) < p) ++b;
  // largest word product must fit 64 bits
  unsigned __int128 tot = 0;
  for (uint32_t j = 0; j < 2 * k - 1; ++j) {
    uint32_t t = std::min<uint32_t>(std::min<uint32_t>(j + 1, 2 * k - 1 - j), k);
    FP_CHECK((uint64_t)j * b < 100, FP_EUNSUPPORTED, "fp_gf_create: product exceeds 64 bits");
    tot += ((unsigned __int128)t * (p - 1) * (p - 1)) << (j * b);
  }
  FP_CHECK(tot < ((unsigned __int128)1 << 64), FP_EUNSUPPORTED,
           "fp_gf_create: GF(%u^%u) product does not fit a 64-bit word", p, k);

  fp_gf g = new (std::nothrow) fp_gf_s();
  FP_CHECK(g != nullptr, FP_ENOMEM, "fp_gf_create: out of host memory");
  g->p = p; g->k = k; g->b = b; g->c = cbits; g->fb = fb; g->order = (uint32_t)order;
  g->elem_bytes = order <= 256 ? 1 : 2;
  g->device = ctx->device;
  // modulus: smallest key sum_{i<k} c_i p^i among monic irreducibles
  for (uint64_t key = 0; key < order; ++key) {
    std::vector<uint32_t> f(k + 1);
    uint64_t x = key;
    for (uint32_t i = 0; i < k; ++i) { f[i] = (uint32_t)(x % p); x /= p; }
    f[k] = 1;
    if (k == 1 || irreducible(f, p)) { g->modulus = f; break; }
  }
  if (g->modulus.empty()) { delete g; set_error("fp_gf_create: no irreducible found"); return FP_EINVAL; }

  // tables
  std::vector<uint64_t> word(order);
  for (uint64_t x = 0; x < order; ++x) {
    uint64_t w = 0, y = x;
    std::vector<uint32_t> cf(k);
    for (uint32_t i = 0; i < k; ++i) { cf[i] = (uint32_t)(y % p); y /= p; }
    for (int i = (int)k - 1; i >= 0; --i) w = (w << b) | cf[i];
    word[x] = w;
  }
  const uint32_t tsz = 1u << (cbits * k);
  const uint32_t cq = (uint32_t)((p - ((1ull << b) % p)) % p);  // -q mod p
  std::vector<uint32_t> L(tsz, 0), H(tsz, 0);
  for (uint32_t idx = 0; idx < tsz; ++idx) {
    std::vector<uint32_t> u(k);
    bool valid = true;
    for (uint32_t i = 0; i < k; ++i) {
      u[i] = (idx >> (i * cbits)) & ((1u << cbits) - 1);
      valid &= u[i] < p;
    }
    if (!valid) continue;
    // L = sum_{i=0}^{k-2} (u_i - q u_{i+1} mod p) X^i  (u = u_0..u_{k-1})
    std::vector<uint32_t> pl(2 * k - 1, 0);
    for (uint32_t i = 0; i + 1 < k; ++i) pl[i] = (u[i] + cq * u[i + 1]) % p;
    L[idx] = spread(poly_rem(pl, g->modulus, p), fb);
    // H = u_{2k-2} X^{2k-2} + sum_{i=k-1}^{2k-3} (u_i - q u_{i+1} mod p) X^i  (u = u_{k-1}..)
    std::vector<uint32_t> ph(2 * k - 1, 0);
    ph[2 * k - 2] = u[k - 1];
    for (uint32_t j = 0; j + 1 < k; ++j) ph[k - 1 + j] = (u[j] + cq * u[j + 1]) % p;
    H[idx] = spread(poly_rem(ph, g->modulus, p), fb);
  }
  g->P = make_redq(p, b, 2 * k - 1);
  cudaError_t e = cudaMalloc(&g->d_word, order * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_L, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_H, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(g->d_word, word.data(), order * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_L, L.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_H, H.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fp_gf_destroy(g);
    return cuda_fail(e, "fp_gf_create tables");
  }
  *out = g;
  return FP_OK;
}

extern "C" void fp_gf_destroy(fp_gf g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->d_word) cudaFree(g->d_word);
  if (g->d_L) cudaFree(g->d_L);
  if (g->d_H) cudaFree(g->d_H);
  delete g;
}

extern "C" fp_status fp_gf_info(fp_gf g, uint32_t* modulus, uint32_t* b, uint32_t* word, uint32_t* elem_bytes) {
  FP_CHECK(g != nullptr, FP_EINVAL, "fp_gf_info: gf is NULL");
  if (modulus)
    for (uint32_t i = 0; i <= g->k; ++i) modulus[i] = g->modulus[i];
  if (b) *b = g->b;
  if (word) *word = FP_WORD_U64;
  if (elem_bytes) *elem_bytes = g->elem_bytes;
  return FP_OK;
}

extern "C" fp_status fp_gf_mul_batched(fp_ctx ctx, fp_gf g, const void* a, const void* b, void* c, size_t count,
                                       void* stream) {
  FP_CHECK(ctx && g, FP_EINVAL, "fp_gf_mul_batched: null ctx or field");
  if (count == 0) return FP_OK;
  FP_CHECK(a && b && c, FP_EINVAL, "fp_gf_mul_batched: null array");
  cudaStream_t st = as_stream(stream);
  const uint32_t tsz = 1u << (g->c * g->k);
  size_t smem = g->order * sizeof(uint64_t) + 2 * tsz * sizeof(uint32_t);
  int grid = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)ctx->num_sms * 4);
  GfDev G{g->d_word, g->d_L, g->d_H, g->order, g->k, g->c, g->fb, 0};
  for (uint32_t i = 0; i < g->k; ++i) G.ones |= 1u << (i * g->fb);
  const bool aligned = ((((uintptr_t)a) | ((uintptr_t)b) | ((uintptr_t)c)) & 15u) == 0;
  // fields with compile-time parameters: full tiles of 4096 pairs (4 per item) on k_gf_mul_fixed
  {
    const uint64_t FITEMS = 256 * 4 * 4;
    const uint64_t fnt = aligned ? count / FITEMS : 0;
    const size_t tb = ((smem + 127) / 128) * 128, smem_f = tb + 6 * FITEMS * g->elem_bytes + 64;
    const int grid_f = (int)std::min<uint64_t>(fnt, (uint64_t)ctx->num_sms * 2);
    bool launched = false;
#define FP_GF_FIXED(PP, KK, E)                                                                                        \
    if (!launched && g->p == PP && g->k == KK && g->b == GfConst<PP, KK>::B && g->c == GfConst<PP, KK>::CB &&       \
        g->fb == GfConst<PP, KK>::FB && fnt) {                                                                         \
      FP_CUDA(cudaFuncSetAttribute(k_gf_mul_fixed<PP, KK, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f)); \
      FP_LAUNCH(ctx, "k_gf_mul_fixed", st, (k_gf_mul_fixed<PP, KK, E><<<grid_f, 256, smem_f, st>>>(                 \
                    (const E*)a, (const E*)b, (E*)c, fnt, (uint32_t)tb, G, ctx->d_err)));                             \
      launched = true;                                                                                                 \
    }
    FP_GF_FIXED(3, 5, uint8_t)
    FP_GF_FIXED(7, 4, uint16_t)
    FP_GF_FIXED(2, 8, uint8_t)
#undef FP_GF_FIXED
    if (launched) {
      FP_CUDA(cudaGetLastError());
      const uint64_t fd = fnt * FITEMS, eb = g->elem_bytes;
      if (fd == count) return FP_OK;
      a = (const uint8_t*)a + fd * eb;
      b = (const uint8_t*)b + fd * eb;
      c = (uint8_t*)c + fd * eb;
      count -= fd;
    }
  }
  // full tiles of 4096 pairs through the bulk-copy loop, the tail per thread
  const uint64_t ITEMS = 256 * 16;
  const uint64_t ntiles = aligned ? count / ITEMS : 0;
  const size_t tbytes = ((smem + 127) / 128) * 128;
  const size_t smem_b = tbytes + 6 * ITEMS * g->elem_bytes + 64;
  const uint64_t done = ntiles * ITEMS;
  if (ntiles) {
    const int grid_b = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 2);
    if (g->elem_bytes == 1) {
      FP_CUDA(cudaFuncSetAttribute(k_gf_mul_bulk<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
      FP_LAUNCH(ctx, "k_gf_mul_bulk", st, k_gf_mul_bulk<uint8_t><<<grid_b, 256, smem_b, st>>>(
                    (const uint8_t*)a, (const uint8_t*)b, (uint8_t*)c, ntiles, (uint32_t)tbytes, G, g->P, ctx->d_err));
    } else {
      FP_CUDA(cudaFuncSetAttribute(k_gf_mul_bulk<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
      FP_LAUNCH(ctx, "k_gf_mul_bulk", st, k_gf_mul_bulk<uint16_t><<<grid_b, 256, smem_b, st>>>(
                    (const uint16_t*)a, (const uint16_t*)b, (uint16_t*)c, ntiles, (uint32_t)tbytes, G, g->P, ctx->d_err));
    }
    FP_CUDA(cudaGetLastError());
    if (done == count) return FP_OK;
  }
  const size_t eb = g->elem_bytes;
  a = (const uint8_t*)a + done * eb;
  b = (const uint8_t*)b + done * eb;
  c = (uint8_t*)c + done * eb;
  count -= done;
  grid = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)ctx->num_sms * 4);
  if (g->elem_bytes == 1) {
    FP_CUDA(cudaFuncSetAttribute(k_gf_mul<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_gf_mul", st, k_gf_mul<uint8_t><<<grid, 256, smem, st>>>((const uint8_t*)a, (const uint8_t*)b,
                                                                              (uint8_t*)c, count, G, g->P, ctx->d_err));
  } else {
    FP_CUDA(cudaFuncSetAttribute(k_gf_mul<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_gf_mul", st, k_gf_mul<uint16_t><<<grid, 256, smem, st>>>((const uint16_t*)a, (const uint16_t*)b,
                                                                               (uint16_t*)c, count, G, g->P, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

namespace fpd {
// Launch the segmented multiply for one field (segments already resident at `segs`).
fp_status gf_launch_segments(fp_ctx ctx, fp_gf g, uint8_t* base, const void* segs, uint32_t nseg, cudaStream_t st) {
  const uint32_t tsz = 1u << (g->c * g->k);
  size_t smem = g->order * sizeof(uint64_t) + 2 * tsz * sizeof(uint32_t);
  GfDev G{g->d_word, g->d_L, g->d_H, g->order, g->k, g->c, g->fb, 0};
  for (uint32_t i = 0; i < g->k; ++i) G.ones |= 1u << (i * g->fb);
  const int grid = (int)std::min<uint32_t>(nseg, (uint32_t)ctx->num_sms * 4);
  if (g->elem_bytes == 1) {
    FP_CUDA(cudaFuncSetAttribute(k_gf_mul_seg<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_gf_mul_seg", st,
              k_gf_mul_seg<uint8_t><<<grid, 256, smem, st>>>(base, (const GfSeg*)segs, nseg, G, g->P, ctx->d_err));
  } else {
    FP_CUDA(cudaFuncSetAttribute(k_gf_mul_seg<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FP_LAUNCH(ctx, "k_gf_mul_seg", st,
              k_gf_mul_seg<uint16_t><<<grid, 256, smem, st>>>(base, (const GfSeg*)segs, nseg, G, g->P, ctx->d_err));
  }
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}
uint32_t gf_elem_bytes(fp_gf g) { return g->elem_bytes; }
uint32_t gf_order(fp_gf g) { return g->order; }
}  // namespace fpd
