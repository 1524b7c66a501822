// GF(p^k) multiplication by Algorithm FGDP (Sec. 6) with n = 1, on the device, in the
// algorithm's order:
//   - table DQT: element index -> u64 word sum_i c_i q^i (one shared-memory lookup);
//   - one word product;
//   - REDQ COMPRESSION: u_i = floor(r/q^i) - p floor(s/q^i), i = 0..2k-2 (no correction);
//   - L[u_0..u_{k-1}] and H[u_{k-1}..u_{2k-2}] (Theorem fgdp), each already reduced modulo
//     the field's modulus, indexed in the binary format sum u_i 2^{c i}, c = ceil(log2 p)
//     (Note on Indexing);
//   - one field addition.
// L and H entries hold the coefficient vector "spread" in 4-bit fields (p <= 7) or 8-bit fields,
// so the field addition is one integer add and a per-field conditional subtraction of p.
// These generic kernels serve every field; GF(2^8), GF(3^5) and GF(7^4) also have word-level
// kernels (k_gf_mul_fixed, below) with the same steps on 32-bit words.
#include <algorithm>
#include <type_traits>
#include <cstring>
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
  uint4* d_img = nullptr;                        // word-level tables (GF(2^8), GF(3^5), GF(7^4))
  uint32_t img_bytes = 0;
  fpd::RedqParams P{};
  // dot product (Algorithm FGDP with n > 1): its own q = 2^bd, nc products per REDQ
  uint32_t bd = 0, nc = 0, gen = 0;              // gen: index of the generator of the log form
  uint64_t* d_word_d = nullptr;                  // [p^k] index form -> word at 2^bd
  uint64_t* d_word_dl = nullptr;                 // [p^k] log form -> word at 2^bd (p^k - 1: zero)
  uint32_t* d_Ld = nullptr;                      // [2^{c k}] L and H at 2^bd
  uint32_t* d_Hd = nullptr;
  uint16_t* d_tolog = nullptr;                   // [p^k] index -> log form
  fpd::RedqParams Pd{};
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

// Field addition of two spread coefficient vectors (fields of fb bits, each < p, 2^(fb-1) >= p):
// one add, then p is taken off every field that reached p -- adding 2^(fb-1) - p to a field
// sets its bit fb-1 exactly when the field is >= p, and no field carries into the next.
__device__ __forceinline__ uint32_t gf_spread_add(uint32_t x, uint32_t y, uint32_t p, uint32_t fb, uint32_t ones) {
  const uint32_t hb = fb - 1;
  const uint32_t t = x + y;
  const uint32_t ge = ((t + ((1u << hb) - p) * ones) >> hb) & ones;
  return t - p * ge;
}

// The last steps of Algorithm FGDP on an accumulated word r: REDQ compression, the two lookups
// and the field addition of their results, returned as a spread coefficient vector (k fields of
// fb bits, each < p).
__device__ __forceinline__ uint32_t gf_redq_spread(uint64_t r, const GfDev& G, const uint32_t* sL,
                                                   const uint32_t* sH, const RedqParams& P) {
  const uint32_t p = P.p, bq = P.b, k = G.k, fb = G.fb, cbits = G.cbits;
  const uint64_t s = divp64(r, P.dv);             // REDQ compression quotient
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
  return gf_spread_add(sL[il], sH[ih], p, fb, G.ones);   // two lookups, one field addition
}

// Index sum_j c_j p^j of a spread coefficient vector.
__device__ __forceinline__ uint32_t gf_spread_index(uint32_t x, uint32_t p, uint32_t k, uint32_t fb) {
  const uint32_t fmask = (1u << fb) - 1u;
  uint32_t idx = 0;
  for (int j = (int)k - 1; j >= 0; --j) idx = idx * p + ((x >> (j * fb)) & fmask);
  return idx;
}

// One product by Algorithm FGDP with n = 1 (see the file comment).
__device__ __forceinline__ uint32_t gf_mul_one(uint32_t xa, uint32_t xb, const GfDev& G, const uint64_t* sw,
                                               const uint32_t* sL, const uint32_t* sH, const RedqParams& P,
                                               uint32_t& bad) {
  bad |= (xa >= G.order) | (xb >= G.order);
  xa = xa < G.order ? xa : 0u;
  xb = xb < G.order ? xb : 0u;
  const uint64_t r = sw[xa] * sw[xb];             // table conversion and the word product
  return gf_spread_index(gf_redq_spread(r, G, sL, sH, P), P.p, G.k, G.fb);
}

template <typename E>
__global__ void __launch_bounds__(256) k_gf_mul(const E* __restrict__ a, const E* __restrict__ b, E* __restrict__ c,
                                                uint64_t count, GfDev G, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
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

// ------------------------------------------------------------------ dot product
//
// Algorithm FGDP with n > 1 (the dot product it is written for).  The element arrays are in
// index or discrete-log form; the word table of the call's form maps an element straight to its
// evaluation at the dot product's own q = 2^bd, so the kernel never sees the form.  Each
// thread accumulates word products while every digit stays below q: after nc products
// (nc (p-1)^2 k < q and the word below 2^64) the word goes through REDQ and the lookups and the
// resulting element, a spread coefficient vector, is added to the thread's running sum in the
// field.  Warps and blocks combine their sums with the same spread addition; a one-block kernel
// adds the per-block sums and writes the result in the call's form.

struct GfDotDev {
  GfDev G;           // word table of the call's form at 2^bd, L and H at 2^bd
  uint32_t nc;       // word products per REDQ
  uint32_t zero;     // the zero element's code in the call's form (invalid codes count as it)
};

template <typename E>
__device__ __forceinline__ void gf_dot_step(uint32_t x, uint32_t y, const GfDotDev& D, const uint64_t* sw,
                                            const uint32_t* sL, const uint32_t* sH, const RedqParams& P,
                                            uint64_t& r, uint32_t& cnt, uint32_t& acc, uint32_t& bad) {
  bad |= (x >= D.G.order) | (y >= D.G.order);
  x = x < D.G.order ? x : D.zero;
  y = y < D.G.order ? y : D.zero;
  r += sw[x] * sw[y];
  if (++cnt == D.nc) {
    acc = gf_spread_add(acc, gf_redq_spread(r, D.G, sL, sH, P), P.p, D.G.fb, D.G.ones);
    r = 0;
    cnt = 0;
  }
}

// Sum of the block's spread vectors; the result is valid in thread 0.
__device__ __forceinline__ uint32_t gf_block_sum(uint32_t acc, uint32_t p, uint32_t fb, uint32_t ones) {
  __shared__ uint32_t wsum[32];
  for (int off = 16; off; off >>= 1) acc = gf_spread_add(acc, __shfl_xor_sync(0xffffffffu, acc, off), p, fb, ones);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  if (lane == 0) wsum[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    acc = lane < nwarps ? wsum[lane] : 0u;
    for (int off = 16; off; off >>= 1) acc = gf_spread_add(acc, __shfl_xor_sync(0xffffffffu, acc, off), p, fb, ones);
  }
  return acc;
}

template <typename E>
__global__ void __launch_bounds__(256) k_gf_dot(const E* __restrict__ a, const E* __restrict__ b, uint64_t n,
                                                GfDotDev D, RedqParams P, uint32_t* __restrict__ partial,
                                                uint32_t* err) {
  extern __shared__ __align__(128) uint8_t dsm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(D.G, dsm, sw, sL, sH);
  uint32_t bad = 0, acc = 0, cnt = 0;
  uint64_t r = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  constexpr uint32_t EPV = 16 / sizeof(E);          // elements per 16-byte vector
  uint64_t done = 0;
  if (((((uintptr_t)a) | ((uintptr_t)b)) & 15u) == 0) {
    const uint64_t nvec = n / EPV;
    const uint4* va = reinterpret_cast<const uint4*>(a);
    const uint4* vb = reinterpret_cast<const uint4*>(b);
    for (uint64_t v = tid; v < nvec; v += stride) {
      const uint4 xa = __ldcs(va + v), xb = __ldcs(vb + v);
      const E* ea = reinterpret_cast<const E*>(&xa);
      const E* eb = reinterpret_cast<const E*>(&xb);
#pragma unroll
      for (uint32_t j = 0; j < EPV; ++j) gf_dot_step<E>(ea[j], eb[j], D, sw, sL, sH, P, r, cnt, acc, bad);
    }
    done = nvec * EPV;
  }
  for (uint64_t i = done + tid; i < n; i += stride) gf_dot_step<E>(a[i], b[i], D, sw, sL, sH, P, r, cnt, acc, bad);
  if (cnt) acc = gf_spread_add(acc, gf_redq_spread(r, D.G, sL, sH, P), P.p, D.G.fb, D.G.ones);
  acc = gf_block_sum(acc, P.p, D.G.fb, D.G.ones);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  if (bad) flag_error(err, ERR_RANGE);
}

// Field sum of the per-block spread vectors, written as one element in the call's form.
template <typename E>
__global__ void __launch_bounds__(256) k_gf_dot_final(const uint32_t* __restrict__ partial, uint32_t nparts,
                                                      E* __restrict__ out, uint32_t p, uint32_t k, uint32_t fb,
                                                      uint32_t ones, const uint16_t* __restrict__ to_log) {
  uint32_t acc = 0;
  for (uint32_t i = threadIdx.x; i < nparts; i += blockDim.x) acc = gf_spread_add(acc, partial[i], p, fb, ones);
  acc = gf_block_sum(acc, p, fb, ones);
  if (threadIdx.x == 0) {
    const uint32_t idx = gf_spread_index(acc, p, k, fb);
    *out = (E)(to_log ? to_log[idx] : idx);
  }
}

// ------------------------------------------------------------------ matrix product
//
// C = A B over GF(p^k) by Algorithm FGDP applied to every entry (each C[r][c] is the dot product
// of row r of A and column c of B; Sec. 6 gives the dot product and names the matrix product as
// its use).  A block computes a 64 x 64 tile of C, each thread 4 x 4 entries.  Tiles of 32 inner
// steps of A and B are staged in shared memory already converted to words (one table lookup per
// element, shared by the 64 entries of C that use it); every entry accumulates word products in
// a 64-bit word for nc steps (the dot product's chunk: every digit below 2^bd, the word below
// 2^64), then takes REDQ, the two lookups and the field addition into its running sum.

static constexpr int GFM_TILE = 64, GFM_KT = 32;

template <typename E>
__global__ void __launch_bounds__(256) k_gf_matmul(const E* __restrict__ A, int lda, const E* __restrict__ B,
                                                   int ldb, E* __restrict__ C, int ldc, int m, int n, int kdim,
                                                   GfDotDev D, RedqParams P, const uint16_t* __restrict__ to_log,
                                                   uint32_t* err) {
  extern __shared__ __align__(128) uint8_t gsm[];
  uint64_t* sw;
  uint32_t *sL, *sH;
  gf_load_tables(D.G, gsm, sw, sL, sH);
  const uint32_t tsz = 1u << (D.G.cbits * D.G.k);
  const size_t tab_bytes = ((D.G.order * sizeof(uint64_t) + 2 * tsz * sizeof(uint32_t)) + 127) & ~(size_t)127;
  uint64_t* sA = reinterpret_cast<uint64_t*>(gsm + tab_bytes);   // [GFM_KT][GFM_TILE]
  uint64_t* sB = sA + GFM_KT * GFM_TILE;                          // [GFM_KT][GFM_TILE]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * GFM_TILE, c0 = blockIdx.x * GFM_TILE;
  uint64_t r[4][4];
  uint32_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { r[i][j] = 0; acc[i][j] = 0; }
  uint32_t bad = 0, cnt = 0;
  const uint32_t order = D.G.order;
  for (int l0 = 0; l0 < kdim; l0 += GFM_KT) {
    __syncthreads();   // the previous tile is no longer read
    for (int e = tid; e < GFM_KT * GFM_TILE; e += 256) {
      {  // A: consecutive threads take consecutive inner steps of a row
        const int l = e % GFM_KT, row = e / GFM_KT;
        uint64_t w = 0;
        if (r0 + row < m && l0 + l < kdim) {
          const uint32_t x = A[(size_t)(r0 + row) * lda + l0 + l];
          bad |= x >= order;
          w = sw[x < order ? x : D.zero];
        }
        sA[l * GFM_TILE + row] = w;
      }
      {  // B: consecutive threads take consecutive columns
        const int col = e % GFM_TILE, l = e / GFM_TILE;
        uint64_t w = 0;
        if (c0 + col < n && l0 + l < kdim) {
          const uint32_t x = B[(size_t)(l0 + l) * ldb + c0 + col];
          bad |= x >= order;
          w = sw[x < order ? x : D.zero];
        }
        sB[l * GFM_TILE + col] = w;
      }
    }
    __syncthreads();
    const int steps = min(GFM_KT, kdim - l0);
    for (int l = 0; l < steps; ++l) {
      uint64_t a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[l * GFM_TILE + ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[l * GFM_TILE + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) r[i][j] += a[i] * b[j];
      if (++cnt == D.nc) {
        cnt = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] = gf_spread_add(acc[i][j], gf_redq_spread(r[i][j], D.G, sL, sH, P), P.p, D.G.fb, D.G.ones);
            r[i][j] = 0;
          }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (cnt) acc[i][j] = gf_spread_add(acc[i][j], gf_redq_spread(r[i][j], D.G, sL, sH, P), P.p, D.G.fb, D.G.ones);
      const int row = r0 + ty + 16 * i, col = c0 + tx + 16 * j;
      if (row < m && col < n) {
        const uint32_t idx = gf_spread_index(acc[i][j], P.p, D.G.k, D.G.fb);
        C[(size_t)row * ldc + col] = (E)(to_log ? to_log[idx] : idx);
      }
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// ------------------------------------------------------------------ word-level fields
//
// GF(2^8), GF(3^5) and GF(7^4) take the steps of Algorithm FGDP (n = 1) with every constant
// fixed at compile time and the data kept in 32-bit registers:
//  * the DQT word of an element (q = 2^b, k digits) fits 32 bits, so the product r is one
//    32 x 32 -> 64-bit multiply;
//  * REDQ compression of r runs on two 32-bit pieces split at digit m.  Since
//    u_i = floor(r / q^i) mod p (Algorithm 2 computes exactly these), the high piece
//    r_hi = floor(r / q^m) gives u_m..u_{2k-2}, and r' = u_m q^m + (r mod q^m) has the same
//    floor(r' / q^i) mod p as r for every i < m (r enters through r_hi mod p = u_m only).
//    Each piece takes one 32-bit division by p: a multiply-high by ceil(2^32 / p), exact
//    below 2^31 (p = 3) and 2^32 / 3 (p = 7), which the pieces stay under;
//  * u_i = (r_i - p s_i) mod q for the base-q digits r_i, s_i of a piece x and s = floor(x/p)
//    (the low b bits of floor(x/q^i) - p floor(s/q^i)), formed for all digits at once: even and
//    odd digits in separate lanes of 2b bits, p q added to every lane so that none borrows;
//  * the split of Theorem fgdp is taken at digit m (the proof holds for any split point): the
//    low table, indexed by u_0..u_m, gives sum_{i<m} mu_i X^i; the high table, indexed by
//    u_m..u_{2k-2}, gives sum_{i>=m} mu_i X^i reduced by the modulus.  The u's are packed into
//    c-bit index fields by merging the odd lanes into the even ones and one multiply that moves
//    every field to the top bits of the word (its cross products fall on distinct bits below the
//    index, so nothing carries into it, or above bit 31);
//  * the field addition of the two parts, in the index representation, is table-driven:
//    GF(2^8) XOR; GF(3^5) one lookup of the coefficient sums (the parts hold their coefficients
//    as base-5 digits, and sums of two residues < 3 never carry); GF(7^4) the sum of the two
//    parts' indices minus 7^(i+1) for each coefficient i whose sum reached 7.
// The tables live in one shared-memory image per field (gfw_image), copied whole into every
// block.  Word tables indexed by a byte are replicated 32 times (entry x of lane l at
// 32 x + l) so that the two random word lookups of a warp never meet a bank conflict.

template <uint32_t P, uint32_t K> struct Gfw;
// GF(2^8): q = 2^4, r < 2^60 (15 digits <= 8).  p divides q, so u_i = floor(r / q^i) mod 2 is bit
// 4i of r (the division by p is a shift, and mu_i = u_i).  Split at m = 8: the low part is
// u_0..u_7 itself (degree <= 7 needs no reduction); the high part is one lookup.
template <> struct Gfw<2, 8> {
  static constexpr uint32_t W = 0, H = 32768, BYTES = H + 128;
  // the dot product's log form: the word table indexed by discrete logarithm (replicated)
  static constexpr uint32_t WL = BYTES, END = WL + 32768;
};
// GF(3^5): q = 2^5, r < 2^45 (9 digits <= 20), m = 5; c = 2 index bits per residue.
template <> struct Gfw<3, 5> {
  static constexpr uint32_t W = 0, L = 32768, H = L + 8192, T = H + 512, BYTES = T + 3200;   // T: 5^5 entries
  // dot product at q = 2^7 (six products per REDQ), after the multiply's tables: word table
  // (replicated as W), L and H with entries as five 6-bit coefficient fields
  static constexpr uint32_t DW = BYTES, DL = DW + 32768, DH = DL + 16384, DOT_END = DH + 1024;
  static constexpr uint32_t DWL = DOT_END, END = DWL + 32768;   // DW indexed by discrete logarithm
};
// GF(7^4): q = 2^8, r < 2^54 (7 digits <= 144), m = 3 = k - 1; c = 3.
template <> struct Gfw<7, 4> {
  static constexpr uint32_t W = 0, L = 16384, H = 32768, CT = 49152, BYTES = CT + 2048;
  // dot product at q = 2^9 (three products per REDQ): word table, L and H with entries as four
  // 8-bit coefficient fields
  static constexpr uint32_t DW = BYTES, DL = DW + 16384, DH = DL + 16384, DOT_END = DH + 16384;
  static constexpr uint32_t DWL = DOT_END, END = DWL + 16384;   // DW indexed by discrete logarithm
};

// bits 0, 4, ..., 28 of w -> bits 0..7: bits 8j and 8j + 4 paired at 8j, then a multiply by
// 2^24 + 2^18 + 2^12 + 2^6 moves pair j to bit 24 + 2j (cross products: distinct bits below 24,
// or 32 and above).
__device__ __forceinline__ uint32_t gfw_gather4(uint32_t w) {
  const uint32_t x = (w & 0x01010101u) | ((w >> 3) & 0x02020202u);
  return (x * 0x01041040u) >> 24;
}

// Dot-product word tables indexed by a byte live in shared memory at a stride of 256 bytes per
// entry (entry x of lane l at byte 256 x + 4 l; half of each row unused), so that one byte
// permutation forms a lookup's whole offset: byte j of w above lane l's 4 l.  gfw_wide_table
// spreads the device image's 32-way replicated table (entry x of lane l at word 32 x + l) into
// that layout, 64 KB.
__device__ __forceinline__ void gfw_wide_table(uint32_t* dst, const uint4* __restrict__ src) {
  const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
  for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) dst[64 * (i >> 5) + (i & 31)] = s32[i];
}
__device__ __forceinline__ uint32_t gfw_wide_lookup(const uint8_t* tab, uint32_t w, uint32_t j, uint32_t lane4) {
  return *reinterpret_cast<const uint32_t*>(tab + __byte_perm(w, lane4, 0x5504u | (j << 4)));
}

// u_i for the six 5-bit digits of x < 2^30, s = floor(x / 3) (GF(3^5) pieces): lanes of 10 bits
// holding digits 0, 2, 4 (even) and 1, 3, 5 (odd); 96 = p q per lane keeps each lane in [3, 127].
// Returned as pairs u_{2j} + 4 u_{2j+1} (each u < 3) at bit 10 j: a lane holds u + 32 j' with the
// multiple of q in its bits 5-6, so the odd lanes shifted down by 3 add onto the even ones without
// touching a u and one mask keeps the pairs.
__device__ __forceinline__ uint32_t gfw_pairs_3(uint32_t x, uint32_t s) {
  constexpr uint32_t ME = 0x01F07C1Fu, CE = 0x06018060u, MO = ME << 5, CO = CE << 5;
  const uint32_t te = ((x & ME) | CE) - 3u * (s & ME);
  const uint32_t to = ((x & MO) | CO) - 3u * (s & MO);
  return (te + (to >> 3)) & 0x00F03C0Fu;
}

// u_i for the four byte digits of x, s = floor(x / 7) (GF(7^4) pieces): lanes of 16 bits, 1792 =
// p q per lane keeps each lane in [7, 2047].  Returned as pairs u_{2j} + 8 u_{2j+1} at bit 16 j
// (the multiples of q sit in bits 8-13 of the lane sum, below the next lane, and are masked off).
__device__ __forceinline__ uint32_t gfw_pairs_7(uint32_t x, uint32_t s) {
  constexpr uint32_t ME = 0x00FF00FFu, CE = 0x07000700u;
  const uint32_t te = ((x & ME) | CE) - 7u * (s & ME);
  const uint32_t to = (((x >> 8) & ME) | CE) - 7u * ((s >> 8) & ME);
  return (te + (to << 3)) & 0x003F003Fu;
}

// One product in GF(2^8): wl = replicated word table + lane, H = high-part table.
__device__ __forceinline__ uint32_t gfw_mul_2_8(uint32_t a, uint32_t b, const uint32_t* wl, const uint8_t* H) {
  const uint64_t r = (uint64_t)wl[a * 32] * wl[b * 32];
  return gfw_gather4((uint32_t)r) ^ H[gfw_gather4((uint32_t)(r >> 32))];
}

// The two table indices of one product in GF(3^5) (REDQ of the word product in SWAR form):
// il from u_0..u_5 (the low part, u_5 q^5 folded in), ih from u_5..u_8 (the high part).
__device__ __forceinline__ void gfw_idx_3_5(uint32_t a, uint32_t b, const uint32_t* wl, uint32_t& il, uint32_t& ih) {
  const uint64_t r = (uint64_t)wl[a * 32] * wl[b * 32];
  const uint32_t lo = (uint32_t)r;
  const uint32_t rh = __funnelshift_r(lo, (uint32_t)(r >> 32), 25);    // digits 5..8
  const uint32_t sh = __umulhi(rh, 0x55555556u);                         // floor(rh / 3)
  const uint32_t rl = (lo & 0x01FFFFFFu) + ((rh - 3u * sh) << 25);       // u_5 q^5 + r mod q^5
  const uint32_t sl = __umulhi(rl, 0x55555556u);
  // pairs (u0,u1) (u2,u3) (u4,u5) at bits 0, 10, 20 -> bits 28, 24, 20; (u5,u6) (u7,u8) at
  // bits 0, 10 -> bits 24, 28
  il = (gfw_pairs_3(rl, sl) * 0x10004001u) >> 20;   // (u4+4u5) + 16 (u2+4u3) + 256 (u0+4u1)
  ih = (gfw_pairs_3(rh, sh) * 0x01040000u) >> 24;   // sum_{t<=3} u_{5+t} 4^t
}

// One product in GF(3^5): L/H entries = sum mu_i 5^i, T maps a sum of two of them to the index.
__device__ __forceinline__ uint32_t gfw_mul_3_5(uint32_t a, uint32_t b, const uint32_t* wl, const uint16_t* L,
                                                const uint16_t* H, const uint8_t* T) {
  uint32_t il, ih;
  gfw_idx_3_5(a, b, wl, il, ih);
  return T[L[il] + H[ih]];
}

// The two table indices of one product in GF(7^4): il from u_0..u_3, ih from u_3..u_6.
__device__ __forceinline__ void gfw_idx_7_4(uint32_t a, uint32_t b, const uint32_t* W, uint32_t& il, uint32_t& ih) {
  const uint64_t r = (uint64_t)W[a] * W[b];
  const uint32_t lo = (uint32_t)r;
  const uint32_t rh = __funnelshift_r(lo, (uint32_t)(r >> 32), 24);    // digits 3..6
  const uint32_t sh = __umulhi(rh, 0x24924925u);                         // floor(rh / 7)
  const uint32_t rl = (lo & 0x00FFFFFFu) + ((rh - 7u * sh) << 24);       // u_3 q^3 + r mod q^3
  const uint32_t sl = __umulhi(rl, 0x24924925u);
  // pairs at bits 0 and 16 -> bits 20 and 26
  il = (gfw_pairs_7(rl, sl) * 0x00100400u) >> 20;   // sum_{t<=3} u_t 8^t
  ih = (gfw_pairs_7(rh, sh) * 0x00100400u) >> 20;   // sum_{t<=3} u_{3+t} 8^t
}

// One product in GF(7^4): W word table, L/H entries = spread (4-bit fields) | index << 16,
// ctl = replicated carry table + lane.
__device__ __forceinline__ uint32_t gfw_mul_7_4(uint32_t a, uint32_t b, const uint32_t* W, const uint32_t* L,
                                                const uint32_t* H, const uint32_t* ctl) {
  uint32_t il, ih;
  gfw_idx_7_4(a, b, W, il, ih);
  const uint32_t x = L[il] + H[ih];
  // bit 4i + 3 of x + 0x1111: coefficient sum i >= 7; the multiply moves those four bits to bits
  // 28..31 (cross products on distinct bits below 28, or above 31)
  const uint32_t g = (((x + 0x1111u) & 0x8888u) * 0x02490000u) >> 28;
  return (x >> 16) - ctl[g * 32];
}

// The products of one 32-bit word of indices (four uint8 or two uint16).  Index checks:
// GF(2^8) has none to make; GF(3^5) flags a byte >= 243 (its lookups stay inside the 256-entry
// table); GF(7^4) flags a uint16 >= 2401 and looks up its low 12 bits.
template <uint32_t P, uint32_t K>
struct Gfw32 {
  const uint8_t* tab;
  uint32_t lane;
  uint32_t bad;
  __device__ __forceinline__ uint32_t word(uint32_t wa, uint32_t wb) {
    using G = Gfw<P, K>;
    if constexpr (P == 7) {
      bad |= wa | ((wa & 0x7FFF7FFFu) + 0x769F769Fu) | wb | ((wb & 0x7FFF7FFFu) + 0x769F769Fu);
      const uint32_t* W = reinterpret_cast<const uint32_t*>(tab + G::W);
      const uint32_t* L = reinterpret_cast<const uint32_t*>(tab + G::L);
      const uint32_t* H = reinterpret_cast<const uint32_t*>(tab + G::H);
      const uint32_t* ctl = reinterpret_cast<const uint32_t*>(tab + G::CT) + lane;
      const uint32_t c0 = gfw_mul_7_4(wa & 0xFFFu, wb & 0xFFFu, W, L, H, ctl);
      const uint32_t c1 = gfw_mul_7_4((wa >> 16) & 0xFFFu, (wb >> 16) & 0xFFFu, W, L, H, ctl);
      return c0 | (c1 << 16);
    } else {
      const uint32_t* wl = reinterpret_cast<const uint32_t*>(tab + G::W) + lane;
      // index byte j by one byte permutation; the four results packed by three
      uint32_t c[4];
      if constexpr (P == 3) {
        // a byte >= 243 has its top bit set and its low 7 bits + 13 >= 128
        bad |= (wa & ((wa & 0x7F7F7F7Fu) + 0x0D0D0D0Du)) | (wb & ((wb & 0x7F7F7F7Fu) + 0x0D0D0D0Du));
        const uint16_t* L = reinterpret_cast<const uint16_t*>(tab + G::L);
        const uint16_t* H = reinterpret_cast<const uint16_t*>(tab + G::H);
        const uint8_t* T = tab + G::T;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          c[j] = gfw_mul_3_5(__byte_perm(wa, 0u, 0x4440u + j), __byte_perm(wb, 0u, 0x4440u + j), wl, L, H, T);
      } else {
        const uint8_t* H = tab + G::H;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          c[j] = gfw_mul_2_8(__byte_perm(wa, 0u, 0x4440u + j), __byte_perm(wb, 0u, 0x4440u + j), wl, H);
      }
      return __byte_perm(__byte_perm(c[0], c[1], 0x0040u), __byte_perm(c[2], c[3], 0x0040u), 0x5410u);
    }
  }
  __device__ __forceinline__ bool any_bad() const {
    return (bad & (P == 7 ? 0x80008000u : P == 3 ? 0x80808080u : 0u)) != 0;
  }
};

// Eight indices of each operand per thread and trip (a 16-byte vector of uint16, an 8-byte one of
// uint8), no staging: the arithmetic per byte is high enough that a few loads in flight per warp
// keep up, and the shared memory goes to the tables, whose one copy serves 32 warps.  Eight per
// trip rather than sixteen keeps the grid's threads within one trip of each other at the end.
static constexpr int GFW_THREADS = 1024;
template <uint32_t P> struct GfwVec { using T = uint2; };
template <> struct GfwVec<7> { using T = uint4; };
template <typename Fn>
__device__ __forceinline__ uint2 gfw_apply(const uint2& x, const uint2& y, Fn&& f) {
  return make_uint2(f(x.x, y.x), f(x.y, y.y));
}
template <typename Fn>
__device__ __forceinline__ uint4 gfw_apply(const uint4& x, const uint4& y, Fn&& f) {
  return make_uint4(f(x.x, y.x), f(x.y, y.y), f(x.z, y.z), f(x.w, y.w));
}
template <uint32_t P, uint32_t K>
__global__ void __launch_bounds__(GFW_THREADS, 2) k_gf_mul_fixed(const typename GfwVec<P>::T* __restrict__ a,
                                                                 const typename GfwVec<P>::T* __restrict__ b,
                                                                 typename GfwVec<P>::T* __restrict__ c, uint64_t nvec,
                                                                 const uint4* __restrict__ image, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  constexpr uint32_t IB = Gfw<P, K>::BYTES;
  for (uint32_t i = threadIdx.x; i < IB / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = image[i];
  __syncthreads();
  Gfw32<P, K> op{sm, threadIdx.x & 31u, 0};
  auto word = [&](uint32_t x, uint32_t y) { return op.word(x, y); };
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if constexpr (P == 2) {
    // the lightest field: two vectors of each operand in flight per thread
    for (; i + stride < nvec; i += 2 * stride) {
      const auto va = a[i], vb = b[i], wa = a[i + stride], wb = b[i + stride];
      c[i] = gfw_apply(va, vb, word);
      c[i + stride] = gfw_apply(wa, wb, word);
    }
  }
  for (; i < nvec; i += stride) c[i] = gfw_apply(a[i], b[i], word);
  if (op.any_bad()) flag_error(err, ERR_RANGE);
}

// GF(2^8) dot product on the word-level multiply (Algorithm FGDP with n > 1; `words` is the word
// table of the call's form, indexed by element index or by discrete logarithm): since
// p | q = 2^4 here, REDQ compression of a word r gives u_i = floor(r / q^i) mod 2 = bit 0 of
// digit i, and bit 0 of a sum of digits is the XOR of their bit 0s, so each thread XORs its
// word products into one 64-bit r (every product is below 2^58; the bits above bit 0 of each
// digit are then meaningless, and unused) and takes REDQ once; the field addition in GF(2^8)
// is XOR too, so the block XOR-reduces and writes its sum as a spread vector (coefficient i at
// bit i fb) for the common final kernel.  No code can be out of range.
__global__ void __launch_bounds__(GFW_THREADS, 2) k_gf_dot_w28(const uint4* __restrict__ a, const uint4* __restrict__ b,
                                                              uint64_t nvec, const uint8_t* __restrict__ ta,
                                                              const uint8_t* __restrict__ tb, uint32_t ntail,
                                                              const uint4* __restrict__ words,
                                                              const uint4* __restrict__ image, uint32_t fb,
                                                              uint32_t* __restrict__ partial) {
  extern __shared__ __align__(128) uint8_t sm[];
  using G = Gfw<2, 8>;
  gfw_wide_table(reinterpret_cast<uint32_t*>(sm), words);   // 64 KB, then the 128-byte H table
  for (uint32_t i = threadIdx.x; i < (G::BYTES - G::H) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm + 65536)[i] = image[G::H / 16 + i];
  __syncthreads();
  const uint32_t lane4 = 4u * (threadIdx.x & 31u);
  const uint8_t* H = sm + 65536;
  // XOR of the word products of four index pairs
  auto word = [&](uint32_t x, uint32_t y) {
    uint64_t t = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) t ^= (uint64_t)gfw_wide_lookup(sm, x, j, lane4) * gfw_wide_lookup(sm, y, j, lane4);
    return t;
  };
  uint64_t r = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nvec; i += stride) {
    const uint4 x = __ldcs(a + i), y = __ldcs(b + i);
    r ^= word(x.x, y.x) ^ word(x.y, y.y) ^ word(x.z, y.z) ^ word(x.w, y.w);
  }
  if (blockIdx.x == 0)   // the last n mod 16 elements
    for (uint32_t i = threadIdx.x; i < ntail; i += blockDim.x)
      r ^= (uint64_t)gfw_wide_lookup(sm, ta[i], 0, lane4) * gfw_wide_lookup(sm, tb[i], 0, lane4);
  uint32_t acc = gfw_gather4((uint32_t)r) ^ H[gfw_gather4((uint32_t)(r >> 32))];
  for (int o = 16; o; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ uint32_t ws[GFW_THREADS / 32];
  if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) t ^= ws[w];
    uint32_t sp = 0;
    for (uint32_t i = 0; i < 8; ++i) sp |= ((t >> i) & 1u) << (i * fb);
    partial[blockIdx.x] = sp;
  }
}

// GF(3^5) and GF(7^4) dot products by Algorithm FGDP with n > 1 on 32-bit words (`words`: the
// word table of the call's form, indexed by element index or by discrete logarithm).
// The dot product has its own q: 2^7 for GF(3^5) (a word product's digits are at most
// 5 (p-1)^2 = 20, six products' at most 120 < 2^7; r < 2^63) and 2^9 for GF(7^4) (digits at
// most 3 * 144 = 432 < 2^9; r < 2^63); every word is below 2^30.  Each thread adds CH = 6 (3)
// word products into a 64-bit r, then takes REDQ compression of r in SWAR form on 32-bit
// pieces, as the multiply does: u_i = floor(r / q^i) mod p for every i, from the digits of a
// piece x and of s = floor(x / p) (u_i = (x_i - p s_i) mod q; lanes of 2 b bits hold
// x_i + p q - p s_i, which stays in [p, (p + 1) q)).  r splits three ways: the top piece r >> 5b
// (GF(3^5)) or r >> 4b (GF(7^4)) gives the top u's; the one digit below it gives the next u
// (floor(r / q^j) = d_j + q floor(r / q^(j+1))); the low piece u_j q^j + r mod q^j gives the
// rest (the same floor(. / q^i) mod p below j).  The low and high parts' reduced coefficients
// come from two tables as wide fields (five 6-bit fields for GF(3^5), four 8-bit fields for
// GF(7^4)) and are added into one 32-bit vector of coefficient sums: the field additions are
// deferred.  A fold keeps each field small and congruent mod p (16 = 1 mod 3: the top two bits
// of a 6-bit field go onto its low four, leaving at most 18, and eight REDQs add at most 4
// each; 8 = 1 mod 7: bits 3-7 of a byte go onto bits 0-2, leaving at most 38, and sixteen REDQs
// add at most 12 each); each field is reduced mod p once, at the end, into the spread form of
// the block sum and the common final kernel.  A code >= p^k reads a zero word, so it counts as
// zero, and sets the range error.

// (u_0 + 4 u_1) at bit 0 and (u_2 + 4 u_3) at bit 14 from the 7-bit digits of x (GF(3^5),
// q = 2^7), s = floor(x / 3): even digits in lanes at 0 and 14, odd digits (x >> 7) likewise.
__device__ __forceinline__ uint32_t gfd_pairs_3(uint32_t x, uint32_t s) {
  constexpr uint32_t ME = 0x001FC07Fu, CE = 0x00600180u, MU = 0x0000C003u;   // CE: 3 q per lane
  const uint32_t te = ((x & ME) | CE) - 3u * (s & ME);
  const uint32_t to = (((x >> 7) & ME) | CE) - 3u * ((s >> 7) & ME);
  return (te & MU) | ((to & MU) << 2);
}

// REDQ of r (GF(3^5), q = 2^7, r < 2^63) and the two lookups: u_5..u_8 from r >> 35, u_4 from
// digit 4 and u_5, u_0..u_3 from u_4 q^4 + r mod q^4; L indexed by (u0 + 4 u1) + 16 (u2 + 4 u3)
// + 256 (u4 + 4 u5), H by (u5 + 4 u6) + 16 (u7 + 4 u8).
__device__ __forceinline__ uint32_t gfd_redq_3_5(uint64_t r, const uint32_t* L, const uint32_t* H) {
  const uint32_t lo = (uint32_t)r, hi = (uint32_t)(r >> 32);
  const uint32_t rhh = hi >> 3;                                          // digits 5..8, < 2^28
  const uint32_t yh = gfd_pairs_3(rhh, __umulhi(rhh, 0x55555556u));
  const uint32_t u5 = yh & 3u;
  const uint32_t t4 = (__funnelshift_r(lo, hi, 28) & 0x7Fu) + (u5 << 7);   // d_4 + q u_5
  const uint32_t u4 = t4 - 3u * __umulhi(t4, 0x55555556u);
  const uint32_t rl = (lo & 0x0FFFFFFFu) + (u4 << 28);                  // < 3 2^28
  const uint32_t yl = gfd_pairs_3(rl, __umulhi(rl, 0x55555556u));
  const uint32_t il = ((yl + (yl >> 10)) & 0xFFu) + ((u4 + 4u * u5) << 8);
  const uint32_t ih = (yh + (yh >> 10)) & 0xFFu;
  return L[il] + H[ih];
}

// (u_0 + 8 u_1) at bit 0 and (u_2 + 8 u_3) at bit 18 from the 9-bit digits of x (GF(7^4),
// q = 2^9), s = floor(x / 7): even digits in lanes at 0 and 18, odd digits (x >> 9) likewise.
__device__ __forceinline__ uint32_t gfd_pairs_7(uint32_t x, uint32_t s) {
  constexpr uint32_t ME = 0x07FC01FFu, CE = 0x38000E00u, MU = 0x001C0007u;   // CE: 7 q per lane
  const uint32_t te = ((x & ME) | CE) - 7u * (s & ME);
  const uint32_t to = (((x >> 9) & ME) | CE) - 7u * ((s >> 9) & ME);
  return (te & MU) | ((to & MU) << 3);
}

// REDQ of r (GF(7^4), q = 2^9, r < 2^63) and the two lookups.  u_4..u_6 from r >> 36; u_3 from
// digit 3 and u_4 (floor(r / q^3) = d_3 + q floor(r / q^4)); the low piece u_3 q^3 + r mod q^3
// gives u_0..u_3.
__device__ __forceinline__ uint32_t gfd_redq_7_4(uint64_t r, const uint32_t* L, const uint32_t* H) {
  const uint32_t lo = (uint32_t)r, hi = (uint32_t)(r >> 32);
  const uint32_t rhh = hi >> 4;                                          // digits 4..6, < 2^27
  const uint32_t yh = gfd_pairs_7(rhh, __umulhi(rhh, 0x24924925u));     // (u4 + 8 u5), u6 at 18
  const uint32_t t3 = (__funnelshift_r(lo, hi, 27) & 0x1FFu) + ((yh & 7u) << 9);
  const uint32_t u3 = t3 - 7u * __umulhi(t3, 0x24924925u);
  const uint32_t rl = (lo & 0x07FFFFFFu) + (u3 << 27);                  // < 7 2^27
  const uint32_t yl = gfd_pairs_7(rl, __umulhi(rl, 0x24924925u));
  const uint32_t il = (yl + (yl >> 12)) & 0xFFFu;                       // u0 + 8 u1 + 64 u2 + 512 u3
  const uint32_t ih = u3 + (((yh + (yh >> 12)) & 0x1FFu) << 3);         // u3 + 8 u4 + 64 u5 + 512 u6
  return L[il] + H[ih];
}

static constexpr int GFD_THREADS = 1024;
template <uint32_t P, uint32_t K>
__global__ void __launch_bounds__(GFD_THREADS, 1) k_gf_dot_wsum(const uint4* __restrict__ a, const uint4* __restrict__ b,
                                                               uint64_t nvec, const void* __restrict__ ta,
                                                               const void* __restrict__ tb, uint32_t ntail,
                                                               const uint4* __restrict__ words,
                                                               const uint4* __restrict__ image, uint32_t fb,
                                                               uint32_t* __restrict__ partial, uint32_t* err) {
  using G = Gfw<P, K>;
  // shared memory: the word table (GF(3^5): spread to 256-byte entries, 64 KB), then L and H
  constexpr uint32_t WB = P == 3 ? 65536u : G::DL - G::DW, DB = G::DOT_END - G::DL;
  constexpr uint32_t FW = P == 3 ? 6u : 8u;                    // bits per coefficient field
  constexpr uint32_t EPV = P == 3 ? 16u : 8u;                  // elements per 16-byte vector
  constexpr uint32_t CH = P == 3 ? 6u : 3u;                    // word products per REDQ
  extern __shared__ __align__(128) uint8_t sm[];
  if constexpr (P == 3) gfw_wide_table(reinterpret_cast<uint32_t*>(sm), words);
  else
    for (uint32_t i = threadIdx.x; i < WB / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = words[i];
  for (uint32_t i = threadIdx.x; i < DB / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm + WB)[i] = image[G::DL / 16 + i];
  __syncthreads();
  const uint32_t* W = reinterpret_cast<const uint32_t*>(sm);
  const uint32_t* L = reinterpret_cast<const uint32_t*>(sm + WB);
  const uint32_t* H = reinterpret_cast<const uint32_t*>(sm + WB + (G::DH - G::DL));
  const uint32_t lane4 = 4u * (threadIdx.x & 31u);
  auto fold = [](uint32_t x) {
    if constexpr (P == 3) return ((x >> 4) & 0x030C30C3u) + (x & 0x0F3CF3CFu);
    else return ((x >> 3) & 0x1F1F1F1Fu) + (x & 0x07070707u);
  };
  auto redq = [&](uint64_t r) {
    if constexpr (P == 3) return gfd_redq_3_5(r, L, H);
    else return gfd_redq_7_4(r, L, H);
  };
  // the word of element e of a vector (as four words); of a code x
  auto eword = [&](const uint32_t* w, uint32_t e) -> uint64_t {
    if constexpr (P == 3) return gfw_wide_lookup(sm, w[e >> 2], e & 3u, lane4);
    else return W[min((e & 1u) ? w[e >> 1] >> 16 : w[e >> 1] & 0xFFFFu, 2401u)];   // >= 2401: a zero word
  };
  auto word = [&](uint32_t x) -> uint64_t {
    if constexpr (P == 3) return gfw_wide_lookup(sm, x, 0, lane4);
    else return W[x];
  };
  // a byte >= 243 has its top bit set and its low 7 bits + 13 >= 128; a uint16 >= 2401 its
  // bit 15 or (low 15 bits + 0x769F) bit 15
  auto check = [](uint32_t x) {
    if constexpr (P == 3) return x & ((x & 0x7F7F7F7Fu) + 0x0D0D0D0Du);
    else return x | ((x & 0x7FFF7FFFu) + 0x769F769Fu);
  };
  uint32_t acc = 0, bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // three vectors per trip: 3 EPV products, eight REDQs of CH products each, then one fold
  for (; i + 2 * stride < nvec; i += 3 * stride) {
    uint4 va[3], vb[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) { va[v] = __ldcs(a + i + v * stride); vb[v] = __ldcs(b + i + v * stride); }
#pragma unroll
    for (int v = 0; v < 3; ++v) bad |= check(va[v].x) | check(va[v].y) | check(va[v].z) | check(va[v].w) |
                                       check(vb[v].x) | check(vb[v].y) | check(vb[v].z) | check(vb[v].w);
#pragma unroll
    for (uint32_t g = 0; g < 3 * EPV / CH; ++g) {
      uint64_t r = 0;
#pragma unroll
      for (uint32_t t = CH * g; t < CH * g + CH; ++t) {
        const uint32_t* wa = reinterpret_cast<const uint32_t*>(&va[t / EPV]);
        const uint32_t* wb = reinterpret_cast<const uint32_t*>(&vb[t / EPV]);
        r += eword(wa, t % EPV) * eword(wb, t % EPV);
      }
      acc += redq(r);
    }
    acc = fold(acc);
  }
  // the rest one product at a time, REDQ after every CH-th
  uint64_t r = 0;
  uint32_t cnt = 0;
  auto push_w = [&](uint64_t wx, uint64_t wy) {
    r += wx * wy;
    if (++cnt == CH) {
      acc = fold(acc + redq(r));
      r = 0;
      cnt = 0;
    }
  };
  for (; i < nvec; i += stride) {
    const uint4 xa = __ldcs(a + i), xb = __ldcs(b + i);
    bad |= check(xa.x) | check(xa.y) | check(xa.z) | check(xa.w) | check(xb.x) | check(xb.y) | check(xb.z) | check(xb.w);
    const uint32_t* wa = reinterpret_cast<const uint32_t*>(&xa);
    const uint32_t* wb = reinterpret_cast<const uint32_t*>(&xb);
#pragma unroll
    for (uint32_t e = 0; e < EPV; ++e) push_w(eword(wa, e), eword(wb, e));
  }
  if (blockIdx.x == 0)   // the last n mod EPV elements, one per thread
    for (uint32_t j = threadIdx.x; j < ntail; j += blockDim.x) {
      uint32_t x, y;
      if constexpr (P == 3) {
        x = static_cast<const uint8_t*>(ta)[j];
        y = static_cast<const uint8_t*>(tb)[j];
        bad |= (x >= 243u || y >= 243u) ? 0x80u : 0u;
      } else {
        x = static_cast<const uint16_t*>(ta)[j];
        y = static_cast<const uint16_t*>(tb)[j];
        bad |= (x >= 2401u || y >= 2401u) ? 0x8000u : 0u;
        x = min(x, 2401u);
        y = min(y, 2401u);
      }
      push_w(word(x), word(y));
    }
  if (cnt) acc = fold(acc + redq(r));
  // each field mod p, into the spread form of the final kernel
  uint32_t sp = 0, ones = 0;
#pragma unroll
  for (uint32_t f = 0; f < K; ++f) {
    sp |= (((acc >> (FW * f)) & ((1u << FW) - 1u)) % P) << (f * fb);
    ones |= 1u << (f * fb);
  }
  sp = gf_block_sum(sp, P, fb, ones);
  if (threadIdx.x == 0) partial[blockIdx.x] = sp;
  if (bad & (P == 3 ? 0x80808080u : 0x80008000u)) flag_error(err, ERR_RANGE);
}

// GF(2^8), GF(3^5), GF(7^4) matrix products on 32-bit words: C = A B with every entry a dot
// product by Algorithm FGDP (Sec. 6), the words and REDQ of the dot products above.  A block
// computes a 64 x 64 tile of C, each thread 4 x 4 entries; tiles of GFMW_KT inner steps of A
// and B are staged in shared memory already as words (one table lookup per element), so an
// inner step is two 16-byte shared loads and 16 multiply-adds of 32-bit words into 64-bit
// accumulators.  GF(3^5) and GF(7^4): REDQ of all 16 accumulators after every CH steps, their
// coefficient vectors added (deferred field additions, folds as in the dot product).  GF(2^8):
// p divides q = 2^4, so u_i = floor(r / q^i) mod 2 is bit 0 of digit i, and bit 0 of a sum of
// digits is the XOR of their bit 0s: the products are XOR-accumulated over the whole inner
// dimension (the bits above bit 0 of each digit are then meaningless, and unused) and the one
// REDQ at the end takes bits 0, 4, ..., 56.  Codes >= p^k read a zero word and set the range error.
static constexpr int GFMW_TILE = 64, GFMW_KT = 32, GFMW_SP = GFMW_TILE + 4;   // row stride: 16-byte rows, fewer conflicts
// the tables a word-level matrix product copies: word table bytes WB (from the form's word table),
// then TB bytes of REDQ tables from image offset TOFF (H at HOFF within them)
template <uint32_t P, uint32_t K> struct GfmwTabs;
template <> struct GfmwTabs<2, 8> {
  static constexpr uint32_t WB = Gfw<2, 8>::H - Gfw<2, 8>::W, TOFF = Gfw<2, 8>::H, TB = 128, HOFF = 0;
};
template <> struct GfmwTabs<3, 5> {
  using G = Gfw<3, 5>;
  static constexpr uint32_t WB = G::DL - G::DW, TOFF = G::DL, TB = G::DOT_END - G::DL, HOFF = G::DH - G::DL;
};
template <> struct GfmwTabs<7, 4> {
  using G = Gfw<7, 4>;
  static constexpr uint32_t WB = G::DL - G::DW, TOFF = G::DL, TB = G::DOT_END - G::DL, HOFF = G::DH - G::DL;
};
template <uint32_t P>
using GfmwElem = typename std::conditional<P == 7, uint16_t, uint8_t>::type;
template <uint32_t P, uint32_t K>
__global__ void __launch_bounds__(256, 2) k_gf_matmul_w(const GfmwElem<P>* __restrict__ A, int lda,
                                                        const GfmwElem<P>* __restrict__ B, int ldb,
                                                        GfmwElem<P>* __restrict__ C, int ldc, int m, int n, int kdim,
                                                        const uint4* __restrict__ words,
                                                        const uint4* __restrict__ image, const uint16_t* __restrict__ to_log,
                                                        uint32_t* err) {
  using T = GfmwTabs<P, K>;
  // shared memory: word table, the REDQ tables, then the A and B tiles
  constexpr uint32_t WB = T::WB, TB = T::TB, TOFF = T::TOFF;
  constexpr uint32_t CH = P == 3 ? 6u : 3u;
  constexpr uint32_t FW = P == 3 ? 6u : 8u;
  constexpr uint32_t ORDER = P == 2 ? 256u : P == 3 ? 243u : 2401u;
  extern __shared__ __align__(128) uint8_t sm[];
  for (uint32_t i = threadIdx.x; i < WB / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = words[i];
  for (uint32_t i = threadIdx.x; i < TB / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm + WB)[i] = image[TOFF / 16 + i];
  const uint32_t* W = reinterpret_cast<const uint32_t*>(sm);
  const uint32_t* L = reinterpret_cast<const uint32_t*>(sm + WB);
  const uint32_t* H = reinterpret_cast<const uint32_t*>(sm + WB + T::HOFF);
  uint32_t* sA = reinterpret_cast<uint32_t*>(sm + WB + TB);   // [GFMW_KT][GFMW_SP]: column l of the A tile
  uint32_t* sB = sA + GFMW_KT * GFMW_SP;                     // [GFMW_KT][GFMW_SP]: row l of the B tile
  const uint32_t lane = threadIdx.x & 31u;
  auto word = [&](uint32_t x) {
    if constexpr (P == 7) return W[min(x, 2401u)];
    else return W[32u * x + lane];                           // replicated table, x < 256
  };
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * GFMW_TILE, c0 = blockIdx.x * GFMW_TILE;
  uint64_t r[4][4];
  uint32_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { r[i][j] = 0; acc[i][j] = 0; }
  uint32_t bad = 0, cnt = 0, chunks = 0;
  auto reduce_all = [&]() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if constexpr (P == 3) acc[i][j] += gfd_redq_3_5(r[i][j], L, H);
        else acc[i][j] += gfd_redq_7_4(r[i][j], L, H);
        r[i][j] = 0;
      }
    if (++chunks == 8) {   // at most 8 REDQs between folds (6-bit fields: 18 + 8 * 4 < 64)
      chunks = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t x = acc[i][j];
          if constexpr (P == 3) acc[i][j] = ((x >> 4) & 0x030C30C3u) + (x & 0x0F3CF3CFu);
          else acc[i][j] = ((x >> 3) & 0x1F1F1F1Fu) + (x & 0x07070707u);
        }
    }
  };
  for (int l0 = 0; l0 < kdim; l0 += GFMW_KT) {
    __syncthreads();   // the tables are in place; the previous tiles are no longer read
    for (int e = tid; e < GFMW_KT * GFMW_TILE; e += 256) {
      {  // A: consecutive threads take consecutive inner steps of a row
        const int l = e % GFMW_KT, row = e / GFMW_KT;
        uint32_t w = 0;
        if (r0 + row < m && l0 + l < kdim) {
          const uint32_t x = A[(size_t)(r0 + row) * lda + l0 + l];
          bad |= x >= ORDER;
          w = word(x);
        }
        sA[l * GFMW_SP + row] = w;
      }
      {  // B: consecutive threads take consecutive columns
        const int col = e % GFMW_TILE, l = e / GFMW_TILE;
        uint32_t w = 0;
        if (c0 + col < n && l0 + l < kdim) {
          const uint32_t x = B[(size_t)(l0 + l) * ldb + c0 + col];
          bad |= x >= ORDER;
          w = word(x);
        }
        sB[l * GFMW_SP + col] = w;
      }
    }
    __syncthreads();
    const int steps = min(GFMW_KT, kdim - l0);
    for (int l = 0; l < steps; ++l) {
      const uint4 av = *reinterpret_cast<const uint4*>(sA + l * GFMW_SP + 4 * ty);
      const uint4 bv = *reinterpret_cast<const uint4*>(sB + l * GFMW_SP + 4 * tx);
      const uint32_t a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if constexpr (P == 2) r[i][j] ^= (uint64_t)a[i] * b[j];
          else r[i][j] += (uint64_t)a[i] * b[j];
        }
      if constexpr (P != 2) {
        if (++cnt == CH) {
          cnt = 0;
          reduce_all();
        }
      }
    }
  }
  if constexpr (P != 2)
    if (cnt) reduce_all();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t idx;
      if constexpr (P == 2) {
        const uint8_t* H8 = reinterpret_cast<const uint8_t*>(L);
        idx = gfw_gather4((uint32_t)r[i][j]) ^ H8[gfw_gather4((uint32_t)(r[i][j] >> 32))];
      } else {
        idx = 0;
#pragma unroll
        for (int f = (int)K - 1; f >= 0; --f) idx = idx * P + ((acc[i][j] >> (FW * f)) & ((1u << FW) - 1u)) % P;
      }
      const int row = r0 + 4 * ty + i, col = c0 + 4 * tx + j;
      if (row < m && col < n) C[(size_t)row * ldc + col] = (GfmwElem<P>)(to_log ? to_log[idx] : idx);
    }
  if (bad) flag_error(err, ERR_RANGE);
}

// Host: the shared-memory image of the word-level tables of the field, empty when the field has
// no word-level kernel.  `word` holds the DQT words, `index`/`rem` the representation helpers.
static std::vector<uint8_t> gfw_image(uint32_t p, uint32_t k, uint32_t b, const std::vector<uint32_t>& modulus,
                                      const std::vector<uint32_t>& antilog) {
  std::vector<uint8_t> img;
  auto digits = [&](uint64_t x) {
    std::vector<uint32_t> c(k);
    for (uint32_t i = 0; i < k; ++i) { c[i] = (uint32_t)(x % p); x /= p; }
    return c;
  };
  auto word = [&](uint64_t x) {
    const std::vector<uint32_t> c = digits(x);
    uint32_t w = 0;
    for (int i = (int)k - 1; i >= 0; --i) w = (w << b) | c[i];
    return w;
  };
  auto index = [&](const std::vector<uint32_t>& c) {
    uint32_t x = 0;
    for (int i = (int)c.size() - 1; i >= 0; --i) x = x * p + c[i];
    return x;
  };
  auto put32 = [&](uint32_t off, uint32_t v) { std::memcpy(img.data() + off, &v, 4); };
  // a log-form code's element: g^e for e < p^k - 1, zero for p^k - 1 (and for invalid codes)
  auto from_log = [&](uint32_t e) { return e < antilog.size() ? antilog[e] : 0u; };
  auto put16 = [&](uint32_t off, uint16_t v) { std::memcpy(img.data() + off, &v, 2); };
  const uint32_t cq = (p - ((1u << b) % p)) % p;   // -q mod p
  uint32_t order = 1;
  for (uint32_t i = 0; i < k; ++i) order *= p;
  if (p == 2 && k == 8 && b == 4) {
    using G = Gfw<2, 8>;
    img.assign(G::BYTES, 0);
    for (uint32_t x = 0; x < 256; ++x)
      for (uint32_t l = 0; l < 32; ++l) put32(G::W + 4 * (32 * x + l), word(x));
    for (uint32_t g = 0; g < 128; ++g) {
      std::vector<uint32_t> ph(2 * k - 1, 0);
      for (uint32_t t = 0; t < 7; ++t) ph[8 + t] = (g >> t) & 1u;
      img[G::H + g] = (uint8_t)index(poly_rem(ph, modulus, p));
    }
    img.resize(G::END, 0);
    for (uint32_t x = 0; x < 256; ++x)
      for (uint32_t l = 0; l < 32; ++l) put32(G::WL + 4 * (32 * x + l), word(from_log(x)));
  } else if (p == 3 && k == 5 && b == 5) {
    using G = Gfw<3, 5>;
    img.assign(G::BYTES, 0);
    for (uint32_t x = 0; x < 256; ++x)
      for (uint32_t l = 0; l < 32; ++l) put32(G::W + 4 * (32 * x + l), x < order ? word(x) : 0u);
    for (uint32_t il = 0; il < 4096; ++il) {   // u_0..u_5 -> sum_{i<5} mu_i X^i (base-5 digits)
      // index layout of gfw_mul_3_5: (u4 + 4 u5) + 16 (u2 + 4 u3) + 256 (u0 + 4 u1)
      uint32_t u[6], v = 0;
      bool ok = true;
      for (uint32_t j = 0; j < 3; ++j) {
        const uint32_t pair = (il >> (4 * (2 - j))) & 15u;
        u[2 * j] = pair & 3u;
        u[2 * j + 1] = pair >> 2;
        ok &= u[2 * j] < p && u[2 * j + 1] < p;
      }
      if (!ok) continue;
      for (uint32_t i = 0, w = 1; i < 5; ++i, w *= 5) v += ((u[i] + cq * u[i + 1]) % p) * w;
      put16(G::L + 2 * il, (uint16_t)v);
    }
    for (uint32_t ih = 0; ih < 256; ++ih) {    // u_5..u_8 -> (sum_{i>=5} mu_i X^i mod P), base-5 digits
      uint32_t u[9] = {0};
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[5 + t] = (ih >> (2 * t)) & 3u; ok &= u[5 + t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> ph(2 * k - 1, 0);
      ph[8] = u[8];
      for (uint32_t i = 5; i < 8; ++i) ph[i] = (u[i] + cq * u[i + 1]) % p;
      const std::vector<uint32_t> r = poly_rem(ph, modulus, p);
      uint32_t v = 0;
      for (uint32_t i = 0, w = 1; i < k; ++i, w *= 5) v += r[i] * w;
      put16(G::H + 2 * ih, (uint16_t)v);
    }
    for (uint32_t x = 0; x < 3125; ++x) {      // base-5 coefficient sums -> index
      uint32_t v = 0, w = 1, y = x;
      for (uint32_t i = 0; i < k; ++i, w *= p, y /= 5) v += ((y % 5) % p) * w;
      img[G::T + x] = (uint8_t)v;
    }
    // dot product at q = 2^7: words with 7-bit digits, L from u_0..u_5 (index
    // (u0 + 4 u1) + 16 (u2 + 4 u3) + 256 (u4 + 4 u5)) and H from u_5..u_8 (index
    // (u5 + 4 u6) + 16 (u7 + 4 u8)), entries as 6-bit coefficient fields
    img.resize(G::DOT_END, 0);
    const uint32_t bd = 7, cqd = (p - ((1u << bd) % p)) % p;
    auto word_d = [&](uint64_t x) {
      const std::vector<uint32_t> c = digits(x);
      uint32_t w = 0;
      for (int i = (int)k - 1; i >= 0; --i) w = (w << bd) | c[i];
      return w;
    };
    auto wide = [&](const std::vector<uint32_t>& c) {
      uint32_t w = 0;
      for (uint32_t i = 0; i < k; ++i) w |= c[i] << (6 * i);
      return w;
    };
    for (uint32_t x = 0; x < 256; ++x)
      for (uint32_t l = 0; l < 32; ++l) put32(G::DW + 4 * (32 * x + l), x < order ? word_d(x) : 0u);
    img.resize(G::END, 0);
    for (uint32_t x = 0; x < 256; ++x)
      for (uint32_t l = 0; l < 32; ++l) put32(G::DWL + 4 * (32 * x + l), word_d(from_log(x)));
    for (uint32_t il = 0; il < 4096; ++il) {
      uint32_t u[6];
      bool ok = true;
      for (uint32_t j = 0; j < 3; ++j) {
        const uint32_t pair = (il >> (4 * j)) & 15u;
        u[2 * j] = pair & 3u;
        u[2 * j + 1] = pair >> 2;
        ok &= u[2 * j] < p && u[2 * j + 1] < p;
      }
      if (!ok) continue;
      std::vector<uint32_t> mu(k);
      for (uint32_t i = 0; i < k; ++i) mu[i] = (u[i] + cqd * u[i + 1]) % p;
      put32(G::DL + 4 * il, wide(mu));
    }
    for (uint32_t ih = 0; ih < 256; ++ih) {
      uint32_t u[9] = {0};
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[5 + t] = (ih >> (2 * t)) & 3u; ok &= u[5 + t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> ph(2 * k - 1, 0);
      ph[8] = u[8];
      for (uint32_t i = 5; i < 8; ++i) ph[i] = (u[i] + cqd * u[i + 1]) % p;
      put32(G::DH + 4 * ih, wide(poly_rem(ph, modulus, p)));
    }
  } else if (p == 7 && k == 4 && b == 8) {
    using G = Gfw<7, 4>;
    img.assign(G::BYTES, 0);
    for (uint32_t x = 0; x < 4096; ++x) put32(G::W + 4 * x, x < order ? word(x) : 0u);
    for (uint32_t il = 0; il < 4096; ++il) {   // u_0..u_3 -> sum_{i<3} mu_i X^i
      uint32_t u[4];
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[t] = (il >> (3 * t)) & 7u; ok &= u[t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> mu(k, 0);
      for (uint32_t i = 0; i < 3; ++i) mu[i] = (u[i] + cq * u[i + 1]) % p;
      uint32_t v = 0;
      for (uint32_t i = 0; i < k; ++i) v |= mu[i] << (4 * i);
      put32(G::L + 4 * il, v | (index(mu) << 16));
    }
    for (uint32_t ih = 0; ih < 4096; ++ih) {   // u_3..u_6 -> sum_{i>=3} mu_i X^i mod P
      uint32_t u[7] = {0};
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[3 + t] = (ih >> (3 * t)) & 7u; ok &= u[3 + t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> ph(2 * k - 1, 0);
      ph[6] = u[6];
      for (uint32_t i = 3; i < 6; ++i) ph[i] = (u[i] + cq * u[i + 1]) % p;
      const std::vector<uint32_t> r = poly_rem(ph, modulus, p);
      uint32_t v = 0;
      for (uint32_t i = 0; i < k; ++i) v |= r[i] << (4 * i);
      put32(G::H + 4 * ih, v | (index(r) << 16));
    }
    for (uint32_t g = 0; g < 16; ++g) {        // 7^(i+1) for every coefficient i that wrapped
      uint32_t v = 0, w = p;
      for (uint32_t i = 0; i < k; ++i, w *= p) v += ((g >> i) & 1u) * w;
      for (uint32_t l = 0; l < 32; ++l) put32(G::CT + 4 * (32 * g + l), v);
    }
    // dot product at q = 2^9: words with 9-bit digits, L from u_0..u_3 and H from u_3..u_6
    // (indices sum_t u 8^t, as above), entries as 8-bit coefficient fields
    img.resize(G::DOT_END, 0);
    const uint32_t bd = 9, cqd = (p - ((1u << bd) % p)) % p;
    auto word_d = [&](uint64_t x) {
      const std::vector<uint32_t> c = digits(x);
      uint32_t w = 0;
      for (int i = (int)k - 1; i >= 0; --i) w = (w << bd) | c[i];
      return w;
    };
    auto wide = [&](const std::vector<uint32_t>& c) {
      uint32_t w = 0;
      for (uint32_t i = 0; i < k; ++i) w |= c[i] << (8 * i);
      return w;
    };
    for (uint32_t x = 0; x < 4096; ++x) put32(G::DW + 4 * x, x < order ? word_d(x) : 0u);
    img.resize(G::END, 0);
    for (uint32_t x = 0; x < 4096; ++x) put32(G::DWL + 4 * x, word_d(from_log(x)));
    for (uint32_t il = 0; il < 4096; ++il) {
      uint32_t u[4];
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[t] = (il >> (3 * t)) & 7u; ok &= u[t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> mu(k, 0);
      for (uint32_t i = 0; i < 3; ++i) mu[i] = (u[i] + cqd * u[i + 1]) % p;
      put32(G::DL + 4 * il, wide(mu));
    }
    for (uint32_t ih = 0; ih < 4096; ++ih) {
      uint32_t u[7] = {0};
      bool ok = true;
      for (uint32_t t = 0; t < 4; ++t) { u[3 + t] = (ih >> (3 * t)) & 7u; ok &= u[3 + t] < p; }
      if (!ok) continue;
      std::vector<uint32_t> ph(2 * k - 1, 0);
      ph[6] = u[6];
      for (uint32_t i = 3; i < 6; ++i) ph[i] = (u[i] + cqd * u[i + 1]) % p;
      put32(G::DH + 4 * ih, wide(poly_rem(ph, modulus, p)));
    }
  }
  return img;
}

// Segmented form for the serving loop: segment s multiplies count[s] pairs at byte offsets
// a/b/c from `base`; one block per segment.
struct GfSeg { uint64_t a, b, c; uint32_t count, pad; };

template <typename E>
__global__ void __launch_bounds__(256) k_gf_mul_seg(uint8_t* base, const GfSeg* __restrict__ segs, uint32_t nseg,
                                                    GfDev G, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
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
  // L and H of Theorem fgdp for q = 2^bq, binary-indexed by (u_0..u_{k-1}) / (u_{k-1}..u_{2k-2})
  auto build_lh = [&](uint32_t bq, std::vector<uint32_t>& L, std::vector<uint32_t>& H) {
    const uint32_t cq = (uint32_t)((p - ((1ull << bq) % p)) % p);  // -q mod p
    L.assign(tsz, 0);
    H.assign(tsz, 0);
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
  };
  std::vector<uint32_t> L, H;
  build_lh(b, L, H);
  g->P = make_redq(p, b, 2 * k - 1);

  // Dot product: the q = 2^bd >= 2^b that lets the most word products accumulate between two
  // REDQ steps: nc k (p-1)^2 < 2^bd (every digit) and nc sum_j t_j (p-1)^2 2^(j bd) < 2^64,
  // t_j = min(j + 1, 2k - 1 - j, k) products meeting at digit j.
  {
    const uint64_t pp = (uint64_t)(p - 1) * (p - 1);
    uint32_t bd = b;
    uint64_t nc = 1;
    for (uint32_t bb = b; bb <= 31; ++bb) {
      if ((uint64_t)(2 * k - 2) * bb >= 64) break;
      unsigned __int128 S = 0;
      for (uint32_t j = 0; j < 2 * k - 1; ++j) {
        const uint32_t t = std::min<uint32_t>(std::min<uint32_t>(j + 1, 2 * k - 1 - j), k);
        S += ((unsigned __int128)t * pp) << (j * bb);
      }
      const uint64_t by_digit = ((1ull << bb) - 1) / (k * pp);
      const unsigned __int128 by_word = ((((unsigned __int128)1) << 64) - 1) / S;
      uint64_t c = std::min<uint64_t>(by_digit, by_word > (1u << 20) ? (uint64_t)(1u << 20) : (uint64_t)by_word);
      if (c > nc) {
        nc = c;
        bd = bb;
      }
    }
    g->bd = bd;
    g->nc = (uint32_t)nc;
  }
  std::vector<uint32_t> Ld, Hd;
  build_lh(g->bd, Ld, Hd);
  g->Pd = make_redq(p, g->bd, 2 * k - 1);
  // Discrete-log form: g^e is written e (0 <= e <= p^k - 2) and zero p^k - 1, with g the
  // smallest index of multiplicative order p^k - 1.
  auto coeffs_of = [&](uint64_t x) {
    std::vector<uint32_t> cf(k);
    for (uint32_t i = 0; i < k; ++i) { cf[i] = (uint32_t)(x % p); x /= p; }
    return cf;
  };
  auto index_of = [&](const std::vector<uint32_t>& cf) {
    uint64_t x = 0;
    for (int i = (int)k - 1; i >= 0; --i) x = x * p + cf[i];
    return x;
  };
  auto fmul = [&](uint64_t x, uint64_t y) {
    const std::vector<uint32_t> cx = coeffs_of(x), cy = coeffs_of(y);
    std::vector<uint32_t> pr(2 * k - 1, 0);
    for (uint32_t i = 0; i < k; ++i)
      for (uint32_t j = 0; j < k; ++j) pr[i + j] = (pr[i + j] + cx[i] * cy[j]) % p;
    return index_of(poly_rem(pr, g->modulus, p));
  };
  auto fpow = [&](uint64_t x, uint64_t e) {
    uint64_t r = 1;
    while (e) {
      if (e & 1) r = fmul(r, x);
      x = fmul(x, x);
      e >>= 1;
    }
    return r;
  };
  {
    const uint64_t nn = order - 1;
    std::vector<uint64_t> primes;
    uint64_t m = nn;
    for (uint64_t d = 2; d * d <= m; ++d)
      if (m % d == 0) {
        primes.push_back(d);
        while (m % d == 0) m /= d;
      }
    if (m > 1) primes.push_back(m);
    g->gen = 1;
    if (nn > 1)
      for (uint64_t cand = 2; cand < order; ++cand) {
        bool full = true;
        for (uint64_t r : primes) full &= fpow(cand, nn / r) != 1;
        if (full) {
          g->gen = (uint32_t)cand;
          break;
        }
      }
  }
  std::vector<uint64_t> word_d(order), word_dl(order, 0);
  std::vector<uint16_t> tolog(order, 0);
  std::vector<uint32_t> antilog(order - 1);
  for (uint64_t x = 0; x < order; ++x) {
    const std::vector<uint32_t> cf = coeffs_of(x);
    uint64_t w = 0;
    for (int i = (int)k - 1; i >= 0; --i) w = (w << g->bd) | cf[i];
    word_d[x] = w;
  }
  {
    uint64_t x = 1;
    for (uint64_t e = 0; e + 1 < order; ++e) {
      word_dl[e] = word_d[x];
      tolog[x] = (uint16_t)e;
      antilog[e] = (uint32_t)x;
      x = fmul(x, g->gen);
    }
    word_dl[order - 1] = 0;
    tolog[0] = (uint16_t)(order - 1);
  }
  cudaError_t e = cudaMalloc(&g->d_word, order * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_L, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_H, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(g->d_word, word.data(), order * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_L, L.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_H, H.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_word_d, order * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_word_dl, order * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_Ld, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_Hd, tsz * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_tolog, order * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(g->d_word_d, word_d.data(), order * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_word_dl, word_dl.data(), order * sizeof(uint64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_Ld, Ld.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_Hd, Hd.data(), tsz * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_tolog, tolog.data(), order * sizeof(uint16_t), cudaMemcpyHostToDevice);
  const std::vector<uint8_t> img = gfw_image(p, k, b, g->modulus, antilog);
  if (e == cudaSuccess && !img.empty()) {
    g->img_bytes = (uint32_t)img.size();
    e = cudaMalloc(&g->d_img, img.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->d_img, img.data(), img.size(), cudaMemcpyHostToDevice);
  }
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
  if (g->d_img) cudaFree(g->d_img);
  if (g->d_word_d) cudaFree(g->d_word_d);
  if (g->d_word_dl) cudaFree(g->d_word_dl);
  if (g->d_Ld) cudaFree(g->d_Ld);
  if (g->d_Hd) cudaFree(g->d_Hd);
  if (g->d_tolog) cudaFree(g->d_tolog);
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

extern "C" fp_status fp_gf_dot_info(fp_gf g, uint32_t* generator, uint32_t* b_dot, uint32_t* chunk) {
  FP_CHECK(g != nullptr, FP_EINVAL, "fp_gf_dot_info: gf is NULL");
  if (generator) *generator = g->gen;
  if (b_dot) *b_dot = g->bd;
  if (chunk) *chunk = g->nc;
  return FP_OK;
}

template <typename E>
static fp_status gf_dot_launch(fp_ctx ctx, fp_gf g, const E* a, const E* b, size_t n, E* out, int form,
                               cudaStream_t st) {
  using namespace fpd;
  constexpr uint64_t EPV = 16 / sizeof(E);   // elements per 16-byte vector
  const bool w28 = g->p == 2 && g->k == 8, w35 = g->p == 3 && g->k == 5, w74 = g->p == 7 && g->k == 4;
  if ((w28 || w35 || w74) && g->d_img && n >= EPV && ((((uintptr_t)a) | ((uintptr_t)b)) & 15u) == 0) {
    // GF(2^8), GF(3^5), GF(7^4), aligned: word-level products, with XOR accumulation (GF(2^8))
    // or three products per REDQ and deferred field additions; the log form reads a word table
    // indexed by discrete logarithm and converts the sum at the end
    const bool lg = form == FP_GF_LOG;
    const uint32_t woff = w28 ? (lg ? Gfw<2, 8>::WL : Gfw<2, 8>::W)
                        : w35 ? (lg ? Gfw<3, 5>::DWL : Gfw<3, 5>::DW) : (lg ? Gfw<7, 4>::DWL : Gfw<7, 4>::DW);
    const uint4* words = g->d_img + woff / 16;
    const void* kern = w28 ? (const void*)k_gf_dot_w28 : w35 ? (const void*)k_gf_dot_wsum<3, 5> : (const void*)k_gf_dot_wsum<7, 4>;
    const size_t smem = w28 ? 65536 + (Gfw<2, 8>::BYTES - Gfw<2, 8>::H)
                      : w35 ? 65536 + (Gfw<3, 5>::DOT_END - Gfw<3, 5>::DL) : Gfw<7, 4>::DOT_END - Gfw<7, 4>::DW;
    const int threads = w28 ? GFW_THREADS : GFD_THREADS;
    FP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const uint64_t nvec = n / EPV;
    const uint64_t want = (nvec + threads - 1) / threads;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->num_sms * std::max(per_sm, 1)));
    fp_status s = ensure_scratch(ctx, (size_t)grid * sizeof(uint32_t), 1, st);
    if (s != FP_OK) return s;
    uint32_t* partial = (uint32_t*)ctx->scratch2;
    const E* ta = a + nvec * EPV;
    const E* tb = b + nvec * EPV;
    const uint32_t ntail = (uint32_t)(n - nvec * EPV);
    if (w28)
      FP_LAUNCH(ctx, "k_gf_dot_w28", st,
                (k_gf_dot_w28<<<grid, GFW_THREADS, smem, st>>>((const uint4*)a, (const uint4*)b, nvec, (const uint8_t*)ta,
                                                                (const uint8_t*)tb, ntail, words, g->d_img, g->fb, partial)));
    else if (w35)
      FP_LAUNCH(ctx, "k_gf_dot_wsum", st,
                (k_gf_dot_wsum<3, 5><<<grid, GFD_THREADS, smem, st>>>((const uint4*)a, (const uint4*)b, nvec, ta, tb, ntail,
                                                                       words, g->d_img, g->fb, partial, ctx->d_err)));
    else
      FP_LAUNCH(ctx, "k_gf_dot_wsum", st,
                (k_gf_dot_wsum<7, 4><<<grid, GFD_THREADS, smem, st>>>((const uint4*)a, (const uint4*)b, nvec, ta, tb, ntail,
                                                                       words, g->d_img, g->fb, partial, ctx->d_err)));
    uint32_t ones = 0;
    for (uint32_t i = 0; i < g->k; ++i) ones |= 1u << (i * g->fb);
    FP_LAUNCH(ctx, "k_gf_dot_final", st,
              (k_gf_dot_final<E><<<1, 256, 0, st>>>(partial, grid, out, g->p, g->k, g->fb, ones,
                                                    lg ? g->d_tolog : nullptr)));
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  const uint32_t tsz = 1u << (g->c * g->k);
  const size_t smem = g->order * sizeof(uint64_t) + 2 * tsz * sizeof(uint32_t);
  GfDotDev D{GfDev{form == FP_GF_LOG ? g->d_word_dl : g->d_word_d, g->d_Ld, g->d_Hd, g->order, g->k, g->c, g->fb, 0},
             g->nc, form == FP_GF_LOG ? g->order - 1 : 0u};
  for (uint32_t i = 0; i < g->k; ++i) D.G.ones |= 1u << (i * g->fb);
  FP_CUDA(cudaFuncSetAttribute(k_gf_dot<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gf_dot<E>, 256, smem));
  const uint64_t per_block = 256ull * (16 / sizeof(E));
  const uint64_t want = (n + per_block - 1) / per_block;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(want, (uint64_t)ctx->num_sms * (uint64_t)std::max(per_sm, 1));
  fp_status s = ensure_scratch(ctx, (size_t)std::max<uint32_t>(grid, 1) * sizeof(uint32_t), 1, st);
  if (s != FP_OK) return s;
  uint32_t* partial = (uint32_t*)ctx->scratch2;
  if (grid)
    FP_LAUNCH(ctx, "k_gf_dot", st, (k_gf_dot<E><<<grid, 256, smem, st>>>(a, b, n, D, g->Pd, partial, ctx->d_err)));
  FP_LAUNCH(ctx, "k_gf_dot_final", st,
            (k_gf_dot_final<E><<<1, 256, 0, st>>>(partial, grid, out, g->p, g->k, g->fb, D.G.ones,
                                                  form == FP_GF_LOG ? g->d_tolog : nullptr)));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

extern "C" fp_status fp_gf_dot(fp_ctx ctx, fp_gf g, const void* a, const void* b, size_t n, void* out, int form,
                               void* stream) {
  FP_CHECK(ctx && g, FP_EINVAL, "fp_gf_dot: null ctx or field");
  FP_CHECK(form == FP_GF_INDEX || form == FP_GF_LOG, FP_EINVAL, "fp_gf_dot: bad form %d", form);
  FP_CHECK(out != nullptr && (n == 0 || (a && b)), FP_EINVAL, "fp_gf_dot: null array");
  FP_CHECK(n < (1ull << 40), FP_EINVAL, "fp_gf_dot: n = %llu above 2^40", (unsigned long long)n);
  cudaStream_t st = as_stream(stream);
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (g->elem_bytes == 1)
    return gf_dot_launch<uint8_t>(ctx, g, (const uint8_t*)a, (const uint8_t*)b, n, (uint8_t*)out, form, st);
  return gf_dot_launch<uint16_t>(ctx, g, (const uint16_t*)a, (const uint16_t*)b, n, (uint16_t*)out, form, st);
}

template <typename E>
static fp_status gf_matmul_launch(fp_ctx ctx, fp_gf g, int m, int n, int kdim, const E* A, int lda, const E* B,
                                  int ldb, E* C, int ldc, int form, cudaStream_t st) {
  using namespace fpd;
  const bool w28 = g->p == 2 && g->k == 8, w35 = g->p == 3 && g->k == 5, w74 = g->p == 7 && g->k == 4;
  if ((w28 || w35 || w74) && g->d_img) {
    // word-level fields: 32-bit words, SWAR REDQ (GF(3^5), GF(7^4)) or XOR accumulation (GF(2^8))
    const bool lg = form == FP_GF_LOG;
    const uint32_t woff = w28 ? (lg ? Gfw<2, 8>::WL : Gfw<2, 8>::W)
                        : w35 ? (lg ? Gfw<3, 5>::DWL : Gfw<3, 5>::DW) : (lg ? Gfw<7, 4>::DWL : Gfw<7, 4>::DW);
    const uint4* words = g->d_img + woff / 16;
    const uint16_t* tl = lg ? g->d_tolog : nullptr;
    const size_t tiles = 2 * (size_t)GFMW_KT * GFMW_SP * sizeof(uint32_t);
    dim3 grid((n + GFMW_TILE - 1) / GFMW_TILE, (m + GFMW_TILE - 1) / GFMW_TILE);
#define FP_GF_MMW(PP, KK)                                                                                         \
    {                                                                                                           \
      const size_t smem = GfmwTabs<PP, KK>::WB + GfmwTabs<PP, KK>::TB + tiles;                                  \
      FP_CUDA(cudaFuncSetAttribute(k_gf_matmul_w<PP, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
      FP_LAUNCH(ctx, "k_gf_matmul_w", st,                                                                       \
                (k_gf_matmul_w<PP, KK><<<grid, 256, smem, st>>>((const GfmwElem<PP>*)A, lda, (const GfmwElem<PP>*)B, \
                                                                ldb, (GfmwElem<PP>*)C, ldc, m, n, kdim, words,      \
                                                                g->d_img, tl, ctx->d_err)));                        \
    }
    if (w28) FP_GF_MMW(2, 8)
    else if (w35) FP_GF_MMW(3, 5)
    else FP_GF_MMW(7, 4)
#undef FP_GF_MMW
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  const uint32_t tsz = 1u << (g->c * g->k);
  const size_t tab = ((g->order * sizeof(uint64_t) + 2 * tsz * sizeof(uint32_t)) + 127) & ~(size_t)127;
  const size_t smem = tab + 2 * (size_t)GFM_KT * GFM_TILE * sizeof(uint64_t);
  GfDotDev D{GfDev{form == FP_GF_LOG ? g->d_word_dl : g->d_word_d, g->d_Ld, g->d_Hd, g->order, g->k, g->c, g->fb, 0},
             g->nc, form == FP_GF_LOG ? g->order - 1 : 0u};
  for (uint32_t i = 0; i < g->k; ++i) D.G.ones |= 1u << (i * g->fb);
  FP_CHECK(smem <= 227 * 1024, FP_EUNSUPPORTED, "fp_gf_matmul: field tables too large for shared memory");
  FP_CUDA(cudaFuncSetAttribute(k_gf_matmul<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((n + GFM_TILE - 1) / GFM_TILE, (m + GFM_TILE - 1) / GFM_TILE);
  FP_LAUNCH(ctx, "k_gf_matmul", st,
            (k_gf_matmul<E><<<grid, 256, smem, st>>>(A, lda, B, ldb, C, ldc, m, n, kdim, D, g->Pd,
                                                     form == FP_GF_LOG ? g->d_tolog : nullptr, ctx->d_err)));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

extern "C" fp_status fp_gf_matmul(fp_ctx ctx, fp_gf g, int m, int n, int k, const void* A, int lda, const void* B,
                                  int ldb, void* C, int ldc, int form, void* stream) {
  FP_CHECK(ctx && g, FP_EINVAL, "fp_gf_matmul: null ctx or field");
  FP_CHECK(form == FP_GF_INDEX || form == FP_GF_LOG, FP_EINVAL, "fp_gf_matmul: bad form %d", form);
  FP_CHECK(m >= 1 && n >= 1 && k >= 1 && m <= (1 << 20) && n <= (1 << 20) && k <= (1 << 20), FP_EINVAL,
           "fp_gf_matmul: m, n, k must lie in [1, 2^20]");
  FP_CHECK(lda >= k && ldb >= n && ldc >= n, FP_EINVAL, "fp_gf_matmul: leading dimension too small");
  FP_CHECK(A && B && C, FP_EINVAL, "fp_gf_matmul: null array");
  cudaStream_t st = fpd::as_stream(stream);
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (g->elem_bytes == 1)
    return gf_matmul_launch<uint8_t>(ctx, g, m, n, k, (const uint8_t*)A, lda, (const uint8_t*)B, ldb, (uint8_t*)C,
                                     ldc, form, st);
  return gf_matmul_launch<uint16_t>(ctx, g, m, n, k, (const uint16_t*)A, lda, (const uint16_t*)B, ldb,
                                    (uint16_t*)C, ldc, form, st);
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
  // word-level fields: whole 16-byte vectors on k_gf_mul_fixed, the rest below
  const uint64_t vbytes = g->elem_bytes == 2 ? 16 : 8;   // eight indices per vector
  if (g->d_img && aligned && count * g->elem_bytes >= vbytes) {
    const uint64_t nvec = count * g->elem_bytes / vbytes;
    bool launched = false;
#define FP_GF_FIXED(PP, KK)                                                                                           \
    if (!launched && g->p == PP && g->k == KK) {                                                                      \
      const size_t smem_f = Gfw<PP, KK>::BYTES;                                                                       \
      FP_CUDA(cudaFuncSetAttribute(k_gf_mul_fixed<PP, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f));  \
      int per_sm = 0;                                                                                                  \
      FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gf_mul_fixed<PP, KK>, GFW_THREADS, smem_f));    \
      const uint64_t want = (nvec + GFW_THREADS - 1) / GFW_THREADS;                                                    \
      const int grid_f = (int)std::min<uint64_t>(want, (uint64_t)ctx->num_sms * (uint64_t)std::max(per_sm, 1));    \
      using VT = typename GfwVec<PP>::T;                                                                              \
      FP_LAUNCH(ctx, "k_gf_mul_fixed", st, (k_gf_mul_fixed<PP, KK><<<grid_f, GFW_THREADS, smem_f, st>>>(            \
                    (const VT*)a, (const VT*)b, (VT*)c, nvec, g->d_img, ctx->d_err)));                                 \
      launched = true;                                                                                                 \
    }
    FP_GF_FIXED(3, 5)
    FP_GF_FIXED(7, 4)
    FP_GF_FIXED(2, 8)
#undef FP_GF_FIXED
    if (launched) {
      FP_CUDA(cudaGetLastError());
      const uint64_t fd = nvec * vbytes / g->elem_bytes, eb = g->elem_bytes;
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
