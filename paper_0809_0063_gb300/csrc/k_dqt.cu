// DQT pack (Eq. dqt), REDQ unpack (Algorithm 2) and the batched polynomial product over F_p
// (Sec. 5): single-word DQT (one word per operand, one word product, one REDQ), blocked FQT
// (Sec. 5.2) for larger degrees, and the plain delayed-reduction baseline (Eq. delayed).
//
// Every kernel stages its contiguous byte tiles through shared memory with 16-byte global
// accesses and runs a grid-stride loop over tiles of 256 items (grid = a multiple of the SM
// count), so HBM traffic is coalesced whatever the number of coefficients per item.
#include <algorithm>
#include <type_traits>

#include "fpdqt_internal.cuh"
#include "stream.cuh"

namespace fpd {

static constexpr int TILE = 256;  // items per tile; one thread per item

// Copy nbytes from global to shared (16-byte vectors when the source is aligned).
__device__ __forceinline__ void stage_in(uint8_t* __restrict__ sm, const uint8_t* __restrict__ g,
                                         uint32_t nbytes) {
  if ((((uintptr_t)g) & 15u) == 0) {
    uint32_t nv = nbytes >> 4;
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x)
      reinterpret_cast<uint4*>(sm)[i] = __ldg(reinterpret_cast<const uint4*>(g) + i);
    for (uint32_t i = (nv << 4) + threadIdx.x; i < nbytes; i += blockDim.x) sm[i] = g[i];
  } else {
    for (uint32_t i = threadIdx.x; i < nbytes; i += blockDim.x) sm[i] = g[i];
  }
}

__device__ __forceinline__ void stage_out(uint8_t* __restrict__ g, const uint8_t* __restrict__ sm,
                                          uint32_t nbytes) {
  if ((((uintptr_t)g) & 15u) == 0) {
    uint32_t nv = nbytes >> 4;
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x)
      reinterpret_cast<uint4*>(g)[i] = reinterpret_cast<const uint4*>(sm)[i];
    for (uint32_t i = (nv << 4) + threadIdx.x; i < nbytes; i += blockDim.x) g[i] = sm[i];
  } else {
    for (uint32_t i = threadIdx.x; i < nbytes; i += blockDim.x) g[i] = sm[i];
  }
}

// Horner evaluation at q = 2^b done with shifts (Sec. 2.1: "the Horner like evaluation of a
// polynomial at q is just a left shift"); the exact integer is then converted to the word.
__device__ __forceinline__ uint64_t pack_bits(const uint8_t* c, uint32_t k, uint32_t b, uint32_t p,
                                              uint32_t& bad) {
  uint64_t w = 0;
  for (int j = (int)k - 1; j >= 0; --j) {
    uint32_t v = c[j];
    bad |= (v >= p);
    w = (w << b) | v;
  }
  return w;
}
// The same for packed values below 2^32 (32-bit shifts).
__device__ __forceinline__ uint32_t pack_bits32(const uint8_t* c, uint32_t k, uint32_t b, uint32_t p, uint32_t& bad) {
  uint32_t w = 0;
  for (int j = (int)k - 1; j >= 0; --j) {
    uint32_t v = c[j];
    bad |= (v >= p);
    w = (w << b) | v;
  }
  return w;
}

// ------------------------------------------------------------------ pack

template <typename W>
__global__ void __launch_bounds__(TILE) k_pack(const uint8_t* __restrict__ coeffs, W* __restrict__ words,
                                               uint64_t count, uint32_t k, uint32_t b, uint32_t p,
                                               uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t ntiles = (count + TILE - 1) / TILE;
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t i0 = t * TILE;
    uint32_t nit = (uint32_t)((count - i0) < (uint64_t)TILE ? (count - i0) : (uint64_t)TILE);
    __syncthreads();
    stage_in(sm, coeffs + i0 * k, nit * k);
    __syncthreads();
    if (threadIdx.x < nit) {
      uint64_t w = pack_bits(sm + threadIdx.x * k, k, b, p, bad);
      words[i0 + threadIdx.x] = WordOps<W>::from_u64(w);
    }
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// ------------------------------------------------------------------ unpack (REDQ)

template <typename W>
__global__ void __launch_bounds__(TILE) k_unpack(const W* __restrict__ words, uint8_t* __restrict__ coeffs,
                                                 uint64_t count, RedqParams P) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector C;
  C.init(P, ptab);
  const uint32_t nd = P.ndig;
  uint64_t ntiles = (count + TILE - 1) / TILE;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t i0 = t * TILE;
    uint32_t nit = (uint32_t)((count - i0) < (uint64_t)TILE ? (count - i0) : (uint64_t)TILE);
    W w = threadIdx.x < nit ? words[i0 + threadIdx.x] : W(0);
    __syncthreads();  // previous tile's stage_out done
    uint8_t* out = sm + threadIdx.x * nd;
    redq_word<W>(w, P, C, [&](uint32_t i, uint32_t mu) { out[i] = (uint8_t)mu; });
    __syncthreads();
    stage_out(coeffs + i0 * nd, sm, nit * nd);
  }
}

// ------------------------------------------------------------------ q = p 2^t (the conclusion)
//
// DQT at q = p 2^t is a Horner evaluation with multiplies.  Its inverse needs no correction: p
// divides q, so -q = 0 mod p and REDQ's residues are the compression values themselves.  The
// compression u_i = floor(r / q^i) - p floor(s / q^i) with s = floor(r / p) uses
// floor(r / q^i) = floor(r / p^i) >> (t i) (nested floors), so with r_i = floor(r / p^i),
// obtained by successive divisions by p (FDIV for FP words, the invariant-divisor multiply for
// integer words), u_i = (r_i >> t i) - p (r_{i+1} >> t i); u_i < p, so 32-bit wrapping suffices.

template <typename W>
__global__ void __launch_bounds__(TILE) k_pack_pq(const uint8_t* __restrict__ coeffs, W* __restrict__ words,
                                                  uint64_t count, uint32_t k, uint64_t q, uint32_t p,
                                                  uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  const uint64_t ntiles = (count + TILE - 1) / TILE;
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t i0 = t * TILE;
    const uint32_t nit = (uint32_t)((count - i0) < (uint64_t)TILE ? (count - i0) : (uint64_t)TILE);
    __syncthreads();
    stage_in(sm, coeffs + i0 * k, nit * k);
    __syncthreads();
    if (threadIdx.x < nit) {
      const uint8_t* c = sm + threadIdx.x * k;
      uint64_t w = 0;
      for (int j = (int)k - 1; j >= 0; --j) {
        const uint32_t v = c[j];
        bad |= v >= p;
        w = w * q + v;
      }
      words[i0 + threadIdx.x] = WordOps<W>::from_u64(w);
    }
  }
  if (bad) flag_error(err, ERR_RANGE);
}

template <typename W>
__global__ void __launch_bounds__(TILE) k_unpack_pq(const W* __restrict__ words, uint8_t* __restrict__ coeffs,
                                                    uint64_t count, RedqParams P, uint32_t t) {
  extern __shared__ __align__(16) uint8_t sm[];
  const uint32_t nd = P.ndig, p = P.p;
  const uint64_t ntiles = (count + TILE - 1) / TILE;
  for (uint64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const uint64_t i0 = tt * TILE;
    const uint32_t nit = (uint32_t)((count - i0) < (uint64_t)TILE ? (count - i0) : (uint64_t)TILE);
    const W w = threadIdx.x < nit ? words[i0 + threadIdx.x] : W(0);
    __syncthreads();  // previous tile's stage_out done
    uint8_t* out = sm + threadIdx.x * nd;
    uint64_t ri = WordOps<W>::to_u64(w);
    for (uint32_t i = 0; i < nd; ++i) {
      const uint64_t rn = WordOps<W>::quot(WordOps<W>::from_u64(ri), P);   // floor(r / p^(i+1))
      const uint32_t sh = t * i;
      const uint32_t a = sh < 64 ? (uint32_t)(ri >> sh) : 0u, bq = sh < 64 ? (uint32_t)(rn >> sh) : 0u;
      out[i] = (uint8_t)(a - p * bq);
      ri = rn;
    }
    __syncthreads();
    stage_out(coeffs + i0 * nd, sm, nit * nd);
  }
}

// ------------------------------------------------------------------ polymul, one word each

// C = A B for small degrees: pack A and B rows (shifts), one word product, REDQ_{ka+kb-1}.
template <typename W>
__global__ void __launch_bounds__(TILE) k_polymul_word(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                       uint8_t* __restrict__ Cout, uint64_t batch, uint32_t ka,
                                                       uint32_t kb, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector C;
  C.init(P, ptab);
  const uint32_t kc = ka + kb - 1;
  uint8_t* sa = sm;
  uint8_t* sb = sm + ((TILE * ka + 15) & ~15u);
  uint8_t* sc = sb + ((TILE * kb + 15) & ~15u);
  uint64_t ntiles = (batch + TILE - 1) / TILE;
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t i0 = t * TILE;
    uint32_t nit = (uint32_t)((batch - i0) < (uint64_t)TILE ? (batch - i0) : (uint64_t)TILE);
    __syncthreads();
    stage_in(sa, A + i0 * ka, nit * ka);
    stage_in(sb, B + i0 * kb, nit * kb);
    __syncthreads();
    W r = W(0);
    if (threadIdx.x < nit) {
      W wa = WordOps<W>::from_u64(pack_bits(sa + threadIdx.x * ka, ka, P.b, P.p, bad));
      W wb = WordOps<W>::from_u64(pack_bits(sb + threadIdx.x * kb, kb, P.b, P.p, bad));
      r = wa * wb;  // Eq. mult: one machine product carries all convolution sums
    }
    uint8_t* out = sc + threadIdx.x * kc;
    redq_word<W>(r, P, C, [&](uint32_t i, uint32_t mu) { out[i] = (uint8_t)mu; });
    __syncthreads();
    stage_out(Cout + i0 * kc, sc, nit * kc);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// The same single-word product on the bulk-copy streaming loop (stream.cuh): 2048 pairs per
// tile, whole tiles moved by the copy engine, double-buffered.
template <typename W>
struct PolymulWordOp {
  static constexpr uint32_t IPT = 8;
  static constexpr uint32_t UNROLL = 2;
  uint32_t ka, kb, kc;
  RedqParams P;
  Corrector C;
  uint32_t bad;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t* b, uint8_t* out) {
    W wa, wb;
    if (sizeof(W) == 4) {
      wa = WordOps<W>::from_u64(pack_bits32(a, ka, P.b, P.p, bad));
      wb = WordOps<W>::from_u64(pack_bits32(b, kb, P.b, P.p, bad));
    } else {
      wa = WordOps<W>::from_u64(pack_bits(a, ka, P.b, P.p, bad));
      wb = WordOps<W>::from_u64(pack_bits(b, kb, P.b, P.p, bad));
    }
    W r = wa * wb;
    redq_word<W>(r, P, C, [&](uint32_t i, uint32_t mu) { out[i] = (uint8_t)mu; });
  }
};

template <typename W>
__global__ void __launch_bounds__(256) k_polymul_word_bulk(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                           uint8_t* __restrict__ Cout, uint64_t ntiles, uint32_t ka,
                                                           uint32_t kb, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  PolymulWordOp<W> op;
  op.ka = ka; op.kb = kb; op.kc = ka + kb - 1; op.P = P; op.bad = 0;
  op.C.init(P, ptab);
  stream_tiles(op, A, B, Cout, ntiles, ka, kb, ka + kb - 1, sm, err);
  if (op.bad) flag_error(err, ERR_RANGE);
}

// Products of small fixed degrees (ka, kb <= 4) in 32-bit words, four pairs per item so that
// every shared-memory access is a whole word: the 4 ka residues of A (and of B) arrive as ka
// words, the 4 kc residues of C leave as kc words.  Per pair: DQT of both operands at q = 2^b
// (Eq. dqt), one 32-bit product, REDQ_kc (Algorithm 2: one division by the invariant p, then
// u_i = ((r >> ib) - p (s >> ib)) mod q) and the correction through the lane-held table (MODE:
// CORR_NONE when p | q, CORR_SHFL3 two residues per lookup, CORR_SHFL2 one).  Residues >= p
// (p < 128) are caught with r | (r + 128 - p) per input word.
// REDQ_KC of a 32-bit word r (Algorithm 2) with the correction through the lane-held table:
// one division s = floor(r / p), u_i = ((r >> ib) - p (s >> ib)) mod q, then mu_i.
template <int KC, int MODE>
__device__ __forceinline__ void redq32_fixed(uint32_t r, uint32_t b, uint32_t p, uint32_t qmask, const DivP& dv,
                                             uint32_t lane_val, uint32_t (&mu)[KC]) {
  const uint32_t s = divp32(r, dv);
  uint32_t u[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) u[i] = ((r >> (i * b)) - p * (s >> (i * b))) & qmask;
  if (MODE == CORR_NONE) {
#pragma unroll
    for (int i = 0; i < KC; ++i) mu[i] = u[i];
  } else if (MODE == CORR_SHFL3) {
#pragma unroll
    for (int i = 0; i + 1 < KC; i += 2) {
      const uint32_t u2 = (i + 2 < KC) ? u[i + 2] : 0u;
      const uint32_t v = __shfl_sync(0xffffffffu, lane_val, u[i] + p * u[i + 1] + p * p * u2);
      mu[i] = v & 0xffu;
      mu[i + 1] = (i + 2 < KC) ? (v >> 8) : u[i + 1];
    }
    if (KC & 1) mu[KC - 1] = u[KC - 1];
  } else {
#pragma unroll
    for (int i = 0; i + 1 < KC; ++i) mu[i] = __shfl_sync(0xffffffffu, lane_val, u[i] + p * u[i + 1]);
    mu[KC - 1] = u[KC - 1];
  }
}

// Up to this many tiles of 2048 pairs the small polynomial products run the direct form (no
// staging); above it, the staged bulk-copy loop.  Measured at 2^20 F_3 pairs of degree 2: 5.45
// vs 6.06 us; at 2^22: 15.8 vs 13.9 us.
static constexpr uint64_t POLY_DIRECT_TILES = 512;

template <int KA, int KB, int MODE>
struct PolySmallOp {
  static constexpr int KC = KA + KB - 1;
  static constexpr uint32_t IPT = 2;
  static constexpr uint32_t UNROLL = 1;
  uint32_t b, p, pk, qmask, lane_val, bad;
  DivP dv;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t* bb, uint8_t* out) {
    uint32_t wa[KA], wb[KB], wc[KC];
#pragma unroll
    for (int i = 0; i < KA; ++i) {
      wa[i] = reinterpret_cast<const uint32_t*>(a)[i];
      bad |= wa[i] | (wa[i] + pk);
    }
#pragma unroll
    for (int i = 0; i < KB; ++i) {
      wb[i] = reinterpret_cast<const uint32_t*>(bb)[i];
      bad |= wb[i] | (wb[i] + pk);
    }
#pragma unroll
    for (int i = 0; i < KC; ++i) wc[i] = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t xa = 0, xb = 0;
#pragma unroll
      for (int i = KA - 1; i >= 0; --i) xa = (xa << b) | ((wa[(j * KA + i) >> 2] >> (8 * ((j * KA + i) & 3))) & 0xffu);
#pragma unroll
      for (int i = KB - 1; i >= 0; --i) xb = (xb << b) | ((wb[(j * KB + i) >> 2] >> (8 * ((j * KB + i) & 3))) & 0xffu);
      uint32_t mu[KC];
      redq32_fixed<KC, MODE>(xa * xb, b, p, qmask, dv, lane_val, mu);
#pragma unroll
      for (int i = 0; i < KC; ++i) wc[(j * KC + i) >> 2] |= mu[i] << (8 * ((j * KC + i) & 3));
    }
#pragma unroll
    for (int i = 0; i < KC; ++i) reinterpret_cast<uint32_t*>(out)[i] = wc[i];
  }
};

// The same item for the paper's own example shape with every parameter fixed: F_3, degree 2 x
// degree 2, q = 16 (the smallest power of two above 3 (p-1)^2 = 12).  Per pair: the three
// coefficient bytes gathered by one byte permutation and packed to nibbles (the DQT at q = 16),
// one product, s = floor(r / 3) by one multiply-high (r < 16^5), all five u_i = (r_i - 3 s_i) mod
// 16 at once in byte lanes (even and odd digits apart, p q = 48 added per lane so none borrows),
// and the correction mu_i = (u_i + c u_{i+1}) mod 3 with c = (-16) mod 3 = 2 for mu_0..mu_3 at
// once in the bytes of one word (sums <= 6, reduced by two per-byte comparisons); mu_4 = u_4.
struct PolyF3Op {
  static constexpr uint32_t IPT = 2;
  static constexpr uint32_t UNROLL = 1;
  uint32_t bad;
  __device__ __forceinline__ static uint32_t pack3(uint32_t t) {   // bytes c0 c1 c2 (< 16) -> c0 + 16 c1 + 256 c2
    return (t & 0xFu) | ((t >> 4) & 0xF0u) | ((t >> 8) & 0xF00u);
  }
  // one product: returns mu_0..mu_3 as bytes; te keeps u_4 in its byte 2
  __device__ __forceinline__ static uint32_t mul(uint32_t ta, uint32_t tb, uint32_t& te) {
    constexpr uint32_t ME = 0x000F0F0Fu, CE = 0x00303030u;
    const uint32_t r = pack3(ta) * pack3(tb);
    const uint32_t s = __umulhi(r, 0x55555556u);
    te = (((r & ME) | CE) - 3u * (s & ME)) & ME;                       // u0 u2 u4
    const uint32_t to = ((((r >> 4) & ME) | CE) - 3u * ((s >> 4) & ME)) & ME;   // u1 u3
    const uint32_t u = __byte_perm(te, to, 0x5140u);                  // u0 u1 u2 u3
    const uint32_t un = __byte_perm(te, to, 0x2514u);                 // u1 u2 u3 u4
    const uint32_t v = u + 2u * un;                                   // bytes <= 6
    const uint32_t ge = (((v + 0x7D7D7D7Du) >> 7) & 0x01010101u) + (((v + 0x7A7A7A7Au) >> 7) & 0x01010101u);
    return v - 3u * ge;
  }
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t* b, uint8_t* out) {
    const uint32_t* pa = reinterpret_cast<const uint32_t*>(a);
    const uint32_t* pb = reinterpret_cast<const uint32_t*>(b);
    const uint32_t a0 = pa[0], a1 = pa[1], a2 = pa[2], b0 = pb[0], b1 = pb[1], b2 = pb[2];
    constexpr uint32_t PK = 0x7D7D7D7Du;                              // 0x01010101 (128 - 3)
    bad |= a0 | (a0 + PK) | a1 | (a1 + PK) | a2 | (a2 + PK) | b0 | (b0 + PK) | b1 | (b1 + PK) | b2 | (b2 + PK);
    uint32_t e0, e1, e2, e3;                                          // byte 2: u_4 = mu_4
    const uint32_t m0 = mul(a0, b0, e0);                              // pair 0: bytes 0-2
    const uint32_t m1 = mul(__byte_perm(a0, a1, 0x5543u), __byte_perm(b0, b1, 0x5543u), e1);   // bytes 3-5
    const uint32_t m2 = mul(__byte_perm(a1, a2, 0x4432u), __byte_perm(b1, b2, 0x4432u), e2);   // bytes 6-8
    const uint32_t m3 = mul(a2 >> 8, b2 >> 8, e3);                    // bytes 9-11
    uint32_t* o = reinterpret_cast<uint32_t*>(out);
    o[0] = m0;
    o[1] = __byte_perm(e0, m1, 0x6542u);                              // mu4(0) mu0..mu2(1)
    o[2] = __byte_perm(__byte_perm(m1, e1, 0x6663u), m2, 0x5410u);    // mu3(1) mu4(1) mu0 mu1(2)
    o[3] = __byte_perm(__byte_perm(m2, e2, 0x6632u), m3, 0x4210u);    // mu2 mu3(2) mu4(2) mu0(3)
    o[4] = __byte_perm(m3, e3, 0x6321u);                              // mu1..mu3(3) mu4(3)
  }
};

__global__ void __launch_bounds__(256) k_polymul_f3(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                    uint8_t* __restrict__ Cout, uint64_t ntiles, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  PolyF3Op op{0};
  stream_tiles(op, A, B, Cout, ntiles, 12, 12, 20, sm, err);
  if (op.bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

// Launched with programmatic dependent launch: the launch of the next kernel on the stream (and
// its blocks' scheduling) overlaps this one, while griddepcontrol.wait, before any global access,
// keeps every read and write after the previous kernel's have completed.
__global__ void __launch_bounds__(256) k_polymul_f3_direct(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                           uint8_t* __restrict__ Cout, uint64_t nitems, uint32_t* err) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  PolyF3Op op{0};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nitems; i += stride)
    op.item(A + i * 12, B + i * 12, Cout + i * 20);
  if (op.bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

template <int KA, int KB, int MODE>
__global__ void __launch_bounds__(256) k_polymul_small(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                       uint8_t* __restrict__ Cout, uint64_t ntiles, RedqParams P,
                                                       uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  PolySmallOp<KA, KB, MODE> op;
  op.b = P.b;
  op.p = P.p;
  op.pk = 0x01010101u * (128u - P.p);
  op.qmask = (1u << P.b) - 1u;
  op.dv = P.dv;
  op.bad = 0;
  Corrector c;
  c.init(P, nullptr);
  op.lane_val = c.lane_val;
  constexpr int KC = KA + KB - 1;
  stream_tiles(op, A, B, Cout, ntiles, 4 * KA, 4 * KB, 4 * KC, sm, err);
  if (op.bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

// The same item, four pairs per thread, read and written in place (no staging): for batches whose
// tiles would give each block only one or two trips of the staged loop, whose load -> compute ->
// store chain per tile is then the whole kernel.
template <int KA, int KB, int MODE>
__global__ void __launch_bounds__(256) k_polymul_small_direct(const uint8_t* __restrict__ A,
                                                              const uint8_t* __restrict__ B, uint8_t* __restrict__ Cout,
                                                              uint64_t nitems, RedqParams P, uint32_t* err) {
  PolySmallOp<KA, KB, MODE> op;
  op.b = P.b;
  op.p = P.p;
  op.pk = 0x01010101u * (128u - P.p);
  op.qmask = (1u << P.b) - 1u;
  op.dv = P.dv;
  op.bad = 0;
  Corrector c;
  c.init(P, nullptr);
  op.lane_val = c.lane_val;
  constexpr int KC = KA + KB - 1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nitems; i += stride)
    op.item(A + i * 4 * KA, B + i * 4 * KB, Cout + i * 4 * KC);
  if (op.bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

template <int KA, int KB>
static bool launch_polymul_small_k(fp_ctx ctx, const uint8_t* A, const uint8_t* B, uint8_t* C, uint64_t ntiles,
                                   const RedqParams& P, cudaStream_t st) {
  constexpr int KC = KA + KB - 1;
  constexpr uint64_t PAIRS = 4 * 256 * 2;   // 4 pairs per item, 256 threads, IPT = 2
  const size_t smem = 2 * PAIRS * (KA + KB + KC) + 64;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 4);
  if (KA == 3 && KB == 3 && P.p == 3 && P.b == 4) {   // the fixed F_3 degree-2 form
    if (ntiles <= POLY_DIRECT_TILES) {
      const uint64_t nitems = ntiles * (PAIRS / 4);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)((nitems + 255) / 256));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      uint32_t* err = ctx->d_err;
      FP_LAUNCH(ctx, "k_polymul_small", st, (cudaLaunchKernelEx(&cfg, k_polymul_f3_direct, A, B, C, nitems, err)));
    } else {
      cudaFuncSetAttribute(k_polymul_f3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_f3<<<grid, 256, smem, st>>>(A, B, C, ntiles, ctx->d_err)));
    }
    return true;
  }
  if (ntiles <= POLY_DIRECT_TILES) {
    // one item (4 pairs) per thread: 512 threads per tile of 2048 pairs
    const uint64_t nitems = ntiles * (PAIRS / 4);
    const int gd = (int)((nitems + 255) / 256);
    switch (P.mode) {
      case CORR_NONE:
        FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small_direct<KA, KB, CORR_NONE><<<gd, 256, 0, st>>>(A, B, C, nitems, P, ctx->d_err)));
        return true;
      case CORR_SHFL3:
        FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small_direct<KA, KB, CORR_SHFL3><<<gd, 256, 0, st>>>(A, B, C, nitems, P, ctx->d_err)));
        return true;
      case CORR_SHFL2:
        FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small_direct<KA, KB, CORR_SHFL2><<<gd, 256, 0, st>>>(A, B, C, nitems, P, ctx->d_err)));
        return true;
      default: return false;
    }
  }
  switch (P.mode) {
    case CORR_NONE:
      cudaFuncSetAttribute(k_polymul_small<KA, KB, CORR_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small<KA, KB, CORR_NONE><<<grid, 256, smem, st>>>(A, B, C, ntiles, P, ctx->d_err)));
      return true;
    case CORR_SHFL3:
      cudaFuncSetAttribute(k_polymul_small<KA, KB, CORR_SHFL3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small<KA, KB, CORR_SHFL3><<<grid, 256, smem, st>>>(A, B, C, ntiles, P, ctx->d_err)));
      return true;
    case CORR_SHFL2:
      cudaFuncSetAttribute(k_polymul_small<KA, KB, CORR_SHFL2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FP_LAUNCH(ctx, "k_polymul_small", st, (k_polymul_small<KA, KB, CORR_SHFL2><<<grid, 256, smem, st>>>(A, B, C, ntiles, P, ctx->d_err)));
      return true;
    default: return false;
  }
}

// Full tiles of 2048 pairs through k_polymul_small when the shape is instantiated (ka = kb in
// {2, 3, 4}), the word is 32-bit, p < 128, the correction is a lane table and the arrays are
// 16-byte aligned; returns the number of pairs done (0 if the path does not apply).
static uint64_t polymul_small(fp_ctx ctx, const uint8_t* A, uint32_t ka, const uint8_t* B, uint32_t kb, uint8_t* C,
                              uint64_t batch, const RedqParams& P, cudaStream_t st) {
  const bool aligned = ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 15u) == 0;
  const uint64_t ntiles = batch / 2048;
  if (!aligned || ntiles == 0 || P.p >= 128 || ka != kb) return 0;
  bool ok = false;
  if (ka == 2) ok = launch_polymul_small_k<2, 2>(ctx, A, B, C, ntiles, P, st);
  else if (ka == 3) ok = launch_polymul_small_k<3, 3>(ctx, A, B, C, ntiles, P, st);
  else if (ka == 4) ok = launch_polymul_small_k<4, 4>(ctx, A, B, C, ntiles, P, st);
  return ok ? ntiles * 2048 : 0;
}

// DQT pack into 32-bit words, K residues per word, four words per item (every shared-memory
// access a whole word): Horner at q = 2^b from the K residue bytes in registers.
template <int K>
struct PackSmallOp {
  static constexpr uint32_t IPT = 4;
  static constexpr uint32_t UNROLL = 1;
  uint32_t b, pk, bad;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t*, uint8_t* out) {
    uint32_t wa[K], wo[4];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      wa[i] = reinterpret_cast<const uint32_t*>(a)[i];
      bad |= wa[i] | (wa[i] + pk);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t x = 0;
#pragma unroll
      for (int i = K - 1; i >= 0; --i) x = (x << b) | ((wa[(j * K + i) >> 2] >> (8 * ((j * K + i) & 3))) & 0xffu);
      wo[j] = x;
    }
    *reinterpret_cast<uint4*>(out) = make_uint4(wo[0], wo[1], wo[2], wo[3]);
  }
};

template <int K>
__global__ void __launch_bounds__(256) k_pack_small(const uint8_t* __restrict__ coeffs, uint32_t* __restrict__ words,
                                                    uint64_t ntiles, uint32_t b, uint32_t p, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  PackSmallOp<K> op;
  op.b = b;
  op.pk = 0x01010101u * (128u - p);
  op.bad = 0;
  stream_tiles(op, coeffs, nullptr, reinterpret_cast<uint8_t*>(words), ntiles, 4 * K, 0, 16, sm, err);
  if (op.bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

// REDQ_ND unpack of 32-bit words, four words per item (ND output words).
template <int ND, int MODE>
struct UnpackSmallOp {
  static constexpr uint32_t IPT = 4;
  static constexpr uint32_t UNROLL = 1;
  uint32_t b, p, qmask, lane_val;
  DivP dv;
  __device__ __forceinline__ void item(const uint8_t* a, const uint8_t*, uint8_t* out) {
    const uint4 w = *reinterpret_cast<const uint4*>(a);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t wc[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) wc[i] = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t mu[ND];
      redq32_fixed<ND, MODE>(ws[j], b, p, qmask, dv, lane_val, mu);
#pragma unroll
      for (int i = 0; i < ND; ++i) wc[(j * ND + i) >> 2] |= mu[i] << (8 * ((j * ND + i) & 3));
    }
#pragma unroll
    for (int i = 0; i < ND; ++i) reinterpret_cast<uint32_t*>(out)[i] = wc[i];
  }
};

template <int ND, int MODE>
__global__ void __launch_bounds__(256) k_unpack_small(const uint32_t* __restrict__ words, uint8_t* __restrict__ coeffs,
                                                      uint64_t ntiles, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  UnpackSmallOp<ND, MODE> op;
  op.b = P.b;
  op.p = P.p;
  op.qmask = (1u << P.b) - 1u;
  op.dv = P.dv;
  Corrector c;
  c.init(P, nullptr);
  op.lane_val = c.lane_val;
  stream_tiles(op, reinterpret_cast<const uint8_t*>(words), nullptr, coeffs, ntiles, 16, 0, 4 * ND, sm, err);
}

// Plain baseline: c_j = sum_i a_i b_{j-i} accumulated without reduction (delayed reduction,
// Eq. delayed: the sums stay far below 2^32), then one reduction mod p per coefficient.
__global__ void __launch_bounds__(TILE) k_polymul_plain_small(const uint8_t* __restrict__ A,
                                                              const uint8_t* __restrict__ B,
                                                              uint8_t* __restrict__ Cout, uint64_t batch,
                                                              uint32_t ka, uint32_t kb, uint32_t p, DivP dv,
                                                              uint32_t* err) {
  extern __shared__ __align__(16) uint8_t sm[];
  const uint32_t kc = ka + kb - 1;
  uint8_t* sa = sm;
  uint8_t* sb = sm + ((TILE * ka + 15) & ~15u);
  uint8_t* sc = sb + ((TILE * kb + 15) & ~15u);
  uint64_t ntiles = (batch + TILE - 1) / TILE;
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t i0 = t * TILE;
    uint32_t nit = (uint32_t)((batch - i0) < (uint64_t)TILE ? (batch - i0) : (uint64_t)TILE);
    __syncthreads();
    stage_in(sa, A + i0 * ka, nit * ka);
    stage_in(sb, B + i0 * kb, nit * kb);
    __syncthreads();
    if (threadIdx.x < nit) {
      const uint8_t* a = sa + threadIdx.x * ka;
      const uint8_t* bb = sb + threadIdx.x * kb;
      uint8_t* out = sc + threadIdx.x * kc;
      for (uint32_t i = 0; i < ka; ++i) bad |= a[i] >= p;
      for (uint32_t i = 0; i < kb; ++i) bad |= bb[i] >= p;
      for (uint32_t j = 0; j < kc; ++j) {
        uint32_t lo = j + 1 > kb ? j + 1 - kb : 0;
        uint32_t hi = j < ka - 1 ? j : ka - 1;
        uint32_t s = 0;
        for (uint32_t i = lo; i <= hi; ++i) s += (uint32_t)a[i] * bb[j - i];
        out[j] = (uint8_t)modp32(s, dv, p);
      }
    }
    __syncthreads();
    stage_out(Cout + i0 * kc, sc, nit * kc);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// Plain baseline for large degrees: one block per pair, one thread per output coefficient.
__global__ void __launch_bounds__(256) k_polymul_plain_big(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                           uint8_t* __restrict__ Cout, uint64_t batch, uint32_t ka,
                                                           uint32_t kb, uint32_t p, DivP dv, uint32_t* err) {
  __shared__ __align__(16) uint8_t sa[1024];
  __shared__ __align__(16) uint8_t sb[1024];
  uint32_t bad = 0;
  const uint32_t kc = ka + kb - 1;
  for (uint64_t t = blockIdx.x; t < batch; t += gridDim.x) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ka; i += blockDim.x) { sa[i] = A[t * ka + i]; bad |= sa[i] >= p; }
    for (uint32_t i = threadIdx.x; i < kb; i += blockDim.x) { sb[i] = B[t * kb + i]; bad |= sb[i] >= p; }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < kc; j += blockDim.x) {
      uint32_t lo = j + 1 > kb ? j + 1 - kb : 0;
      uint32_t hi = j < ka - 1 ? j : ka - 1;
      uint32_t s = 0;
      for (uint32_t i = lo; i <= hi; ++i) s += (uint32_t)sa[i] * sb[j - i];
      Cout[t * kc + j] = (uint8_t)modp32(s, dv, p);
    }
  }
  if (bad) flag_error(err, ERR_RANGE);
}

__global__ void __launch_bounds__(256) k_polymul_fqt(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                     uint8_t* __restrict__ Cout, uint64_t batch, uint32_t ka,
                                                     uint32_t kb, uint32_t d1, RedqParams P, uint32_t* err) {
  __shared__ uint64_t wa[1024];
  __shared__ uint64_t wb[1024];
  __shared__ uint8_t res[4096 + 64];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector C;
  C.init(P, ptab);
  uint32_t bad = 0;
  const uint32_t kc = ka + kb - 1;
  for (uint64_t t = blockIdx.x; t < batch; t += gridDim.x)
    fqt_block_product(A + t * ka, B + t * kb, Cout + t * kc, ka, kb, d1, P, C, wa, wb, res, bad);
  if (bad) flag_error(err, ERR_RANGE);
}

// Largest FQT block size d+1 whose accumulated u64 output word stays exact: digit bound
// min(#blocks) (d+1) (p-1)^2 < q = 2^b, 2d+1 digits below 2^64, shared buffers large enough.
bool fqt_params(uint32_t p, uint32_t ka, uint32_t kb, uint32_t* d1_out, uint32_t* b_out) {
  uint32_t best_d1 = 0, best_b = 0;
  for (uint32_t d1 = 1; d1 <= 32; ++d1) {
    uint32_t na = (ka + d1 - 1) / d1, nb = (kb + d1 - 1) / d1;
    uint64_t nterms = na < nb ? na : nb;
    uint64_t D = nterms * d1 * (uint64_t)(p - 1) * (p - 1);
    uint32_t b = 1;
    while ((1ull << b) <= D || (1ull << b) < p) ++b;
    unsigned __int128 tot = 0;
    bool ok = true;
    for (uint32_t j = 0; j < 2 * d1 - 1 && ok; ++j) {
      if ((uint64_t)j * b >= 100) { ok = false; break; }
      tot += (unsigned __int128)D << (j * b);
      if (tot >> 64) ok = false;
    }
    if (!ok) break;
    if (na > 1024 || nb > 1024 || na + nb - 1 > 2048 || (na + nb - 1) * (2 * d1 - 1) > 4096) continue;
    best_d1 = d1;
    best_b = b;
  }
  *d1_out = best_d1;
  *b_out = best_b;
  return best_d1 >= 1;
}

// ------------------------------------------------------------------ Karatsuba FQT

// Karatsuba version of the blocked FQT (Sec. 5.2; the Karatsuba timings of Fig. pmkara).  The
// operands' word polynomials (blocks of d+1 coefficients in u64 words at q = 2^b, exactly as in
// the blocked FQT) are zero-padded to N = m 2^L words and split L times into low half, high half
// and their sum, giving T = 3^L leaf polynomials of m words each; the leaf products are
// recombined by R = P0 + X^c (P2 - P0 - P1) + X^{2c} P1.  Every step is in Z / 2^64, and
// Karatsuba's identity holds in any commutative ring, so each output word is the same integer
// as the schoolbook sum, which the blocked FQT's digit bound keeps below 2^64: REDQ and the
// overlap of the blocks are unchanged.
struct KaraShape {
  uint32_t d1, L, m, N, T;
};

constexpr uint32_t KARA_PADL = 4;   // zero words below each right-hand leaf (the window reads down to -4)
constexpr uint32_t KARA_PADS = 8;   // zero words per right-hand leaf in all (reads go up to m + 2)

// Shared memory of k_polymul_kara, in bytes: levels 0 (2N words), the leaves of A (T m) and of
// B (T (m + 8)), the leaf products (2 T m), then the nw (2d + 1) REDQ residues.
static size_t kara_smem_bytes(const KaraShape& S, uint32_t nw) {
  const size_t words = 2 * (size_t)S.N + (size_t)S.T * S.m + (size_t)S.T * (S.m + KARA_PADS) + 2 * (size_t)S.T * S.m;
  return words * 8 + (size_t)nw * (2 * S.d1 - 1);
}

__global__ void __launch_bounds__(256) k_polymul_kara(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                                      uint8_t* __restrict__ Cout, uint64_t batch, uint32_t ka,
                                                      uint32_t kb, KaraShape S, RedqParams P, uint32_t* err) {
  extern __shared__ __align__(16) uint64_t ksm[];
  __shared__ uint8_t ptab[1024];
  fill_pair_table(ptab, P);
  __syncthreads();
  Corrector C;
  C.init(P, ptab);
  const uint32_t m = S.m, T = S.T, N = S.N, L = S.L, d1 = S.d1;
  const uint32_t SE = m + KARA_PADS;
  uint64_t* wa = ksm;                               // level 0 of A and B: [N] each
  uint64_t* wb = wa + N;
  uint64_t* ea = wb + N;                            // leaves of A: [T][m]
  uint64_t* eb = ea + (size_t)T * m;                // leaves of B: [T][m + 8], values from word 4
  uint64_t* xs = eb + (size_t)T * SE;               // [T][2m] leaf products (evaluation scratch before)
  uint64_t* ys = ea;                                // interpolation scratch (ea, eb are dead by then)
  uint8_t* res = (uint8_t*)(xs + 2 * (size_t)T * m);
  const uint32_t na = (ka + d1 - 1) / d1, nb = (kb + d1 - 1) / d1;
  const uint32_t nw = na + nb - 1, kc = ka + kb - 1;
  const uint32_t G = (2 * m + 2) / 4;               // groups of four output words per leaf product
  const uint32_t GH = (G + 1) / 2;                  // work items per leaf: groups g and g + GH
  uint32_t bad = 0;
  for (uint64_t t = blockIdx.x; t < batch; t += gridDim.x) {
    __syncthreads();
    fqt_pack(A + t * ka, ka, d1, N, P, wa, bad);
    fqt_pack(B + t * kb, kb, d1, N, P, wb, bad);
    __syncthreads();
    // Evaluation.  Level l holds 3^l segments of h = m 2^(L-l) words; segment s is the low half
    // (s mod 3 = 0), the high half (1) or the sum of both halves (2) of segment s / 3 of level
    // l - 1.  Levels with L - l even live in ea / eb, the others in xs (A) and xs + T m (B).
    uint32_t nseg = 1;
    for (uint32_t l = 1; l <= L; ++l) {
      const uint32_t h = m << (L - l);
      nseg *= 3;
      const uint64_t* sa = l == 1 ? wa : (((L - l + 1) & 1) ? xs : ea);
      const uint64_t* sb = l == 1 ? wb : (((L - l + 1) & 1) ? xs + (size_t)T * m : eb);
      uint64_t* da = ((L - l) & 1) ? xs : ea;
      uint64_t* db = ((L - l) & 1) ? xs + (size_t)T * m : eb;
      const bool last = l == L;
      // u / h = umulhi(u, ceil(2^32 / h)), exact for u h < 2^32 (the multiplier needs h > 1)
      const uint32_t mh = h > 1 ? 0xffffffffu / h + 1u : 0u;
      for (uint32_t u = threadIdx.x; u < nseg * h; u += blockDim.x) {
        const uint32_t sg = h > 1 ? __umulhi(u, mh) : u, j = u - sg * h;
        const uint32_t par = sg / 3, dg = sg - par * 3;
        const uint32_t src = par * 2 * h + (dg == 1 ? h : 0) + j;
        uint64_t va = sa[src], vb = sb[src];
        if (dg == 2) {
          va += sa[src + h];
          vb += sb[src + h];
        }
        da[u] = va;
        db[last ? sg * SE + KARA_PADL + j : u] = vb;
      }
      if (last)
        for (uint32_t u = threadIdx.x; u < T * KARA_PADS; u += blockDim.x) {
          const uint32_t sg = u / KARA_PADS, r = u - sg * KARA_PADS;
          eb[sg * SE + (r < KARA_PADL ? r : m + r)] = 0;
        }
      __syncthreads();
    }
    // Leaf products, four consecutive output words 4g..4g+3 per pass over a sliding window of
    // B's leaf (w_r = b[o0 + r - i]), four steps per round (eight shared loads per sixteen word
    // products).  Group g runs min(m - 1, 4g + 3) - max(0, 4g - m + 1) + 1 steps, about 4g + 4
    // for g < G / 2 and 2m - 4g after, so work item u = gp T + leaf takes groups gp and gp + GH
    // (about m + 4 steps in all) and the lanes of a warp, sharing gp or spanning a few
    // neighbouring values, run each pass for nearly the same number of steps.  The launch gives
    // the block T GH threads (whole warps, 128 to 256), so small products take one round.
    const uint32_t mt = 0xffffffffu / T + 1u;       // u / T = umulhi(u, mt) (T >= 3, u T < 2^32)
    for (uint32_t u = threadIdx.x; u < T * GH; u += blockDim.x) {
      const uint32_t gp = __umulhi(u, mt), leaf = u - gp * T;
      const uint64_t* a = ea + (size_t)leaf * m;
      const uint64_t* bq = eb + (size_t)leaf * SE + KARA_PADL;
      uint64_t* out = xs + 2 * (size_t)leaf * m;
      const int no = 2 * (int)m - 1;
      for (uint32_t g = gp; g < G; g += GH) {
        const int o0 = 4 * (int)g;
        const int ilo = max(0, o0 - (int)m + 1), ihi = min((int)m - 1, o0 + 3);
        uint64_t w0 = bq[o0 - ilo], w1 = bq[o0 + 1 - ilo], w2 = bq[o0 + 2 - ilo], w3 = bq[o0 + 3 - ilo];
        uint64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        int i = ilo;
        for (; i + 3 <= ihi; i += 4) {
          const uint64_t a0 = a[i], a1 = a[i + 1], a2 = a[i + 2], a3 = a[i + 3];
          const uint64_t v1 = bq[o0 - i - 1], v2 = bq[o0 - i - 2], v3 = bq[o0 - i - 3], v4 = bq[o0 - i - 4];
          c0 += a0 * w0 + a1 * v1 + a2 * v2 + a3 * v3;
          c1 += a0 * w1 + a1 * w0 + a2 * v1 + a3 * v2;
          c2 += a0 * w2 + a1 * w1 + a2 * w0 + a3 * v1;
          c3 += a0 * w3 + a1 * w2 + a2 * w1 + a3 * w0;
          w3 = v1;
          w2 = v2;
          w1 = v3;
          w0 = v4;
        }
        for (; i <= ihi; ++i) {
          const uint64_t av = a[i];
          c0 += av * w0;
          c1 += av * w1;
          c2 += av * w2;
          c3 += av * w3;
          w3 = w2;
          w2 = w1;
          w1 = w0;
          w0 = bq[o0 - i - 1];
        }
        if (o0 < no) out[o0] = c0;
        if (o0 + 1 < no) out[o0 + 1] = c1;
        if (o0 + 2 < no) out[o0 + 2] = c2;
        if (o0 + 3 < no) out[o0 + 3] = c3;
      }
    }
    __syncthreads();
    // Interpolation.  Parent u of level l - 1 from its children 3u, 3u+1, 3u+2 of level l
    // (products of 2c - 1 words at stride 2c, c = m 2^(L-l)): R = P0 + X^c (P2 - P0 - P1) +
    // X^(2c) P1, 4c - 1 words at stride 4c.  Level k lives in xs when L - k is even, else in ys.
    uint32_t npar = T;
    for (uint32_t l = L; l >= 1; --l) {
      const uint32_t c = m << (L - l);
      npar /= 3;
      const uint64_t* src = ((L - l) & 1) ? ys : xs;
      uint64_t* dst = ((L - l + 1) & 1) ? ys : xs;
      const uint32_t len = 4 * c - 1;
      const uint32_t ml = 0xffffffffu / len + 1u;   // u / len = umulhi(u, ml) (len >= 3, u len < 2^32)
      for (uint32_t u = threadIdx.x; u < npar * len; u += blockDim.x) {
        const uint32_t par = __umulhi(u, ml), x = u - par * len;
        const uint64_t* P0 = src + 6 * (size_t)c * par;
        const uint64_t* P1 = P0 + 2 * c;
        const uint64_t* P2 = P1 + 2 * c;
        uint64_t r = 0;
        if (x < 2 * c - 1) r += P0[x];
        if (x >= c && x < 3 * c - 1) r += P2[x - c] - P0[x - c] - P1[x - c];
        if (x >= 2 * c) r += P1[x - 2 * c];
        dst[4 * (size_t)c * par + x] = r;
      }
      __syncthreads();
    }
    const uint64_t* root = (L & 1) ? ys : xs;
    fqt_reduce_product([&](uint32_t o) { return root[o]; }, nw, kc, d1, P, C, res, Cout + t * kc);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

// Karatsuba shape for ka x kb coefficients: the blocked FQT's block size and q (the same digit
// bound, see above), and the depth L >= 1 with the least estimated instruction count -- about 4
// per word product (three IMADs, half a shared load), 15 per evaluated word of each operand and
// 20 per interpolated word -- whose shared memory fits in 200 KB.
bool kara_params(uint32_t p, uint32_t ka, uint32_t kb, KaraShape* S, uint32_t* b_out, size_t* smem_out) {
  uint32_t d1 = 0, b = 0;
  if (!fqt_params(p, ka, kb, &d1, &b)) return false;
  const uint32_t na = (ka + d1 - 1) / d1, nb = (kb + d1 - 1) / d1, n0 = std::max(na, nb);
  double best = -1.0;
  for (uint32_t L = 1; L <= 8; ++L) {
    KaraShape c;
    c.d1 = d1;
    c.L = L;
    c.m = (n0 + (1u << L) - 1) >> L;
    c.N = c.m << L;
    c.T = 1;
    for (uint32_t l = 0; l < L; ++l) c.T *= 3;
    const size_t smem = kara_smem_bytes(c, na + nb - 1);
    if (smem > 200 * 1024) break;
    double ev = 0.0, ip = 0.0, t3 = 1.0;
    for (uint32_t l = 1; l <= L; ++l) {
      const double h = (double)(c.m << (L - l));
      ip += t3 * (4.0 * h - 1.0);
      t3 *= 3.0;
      ev += t3 * h;
    }
    const double cost = 4.0 * c.T * (double)c.m * c.m + 30.0 * ev + 20.0 * ip;
    if (best < 0.0 || cost < best) {
      best = cost;
      *S = c;
      *smem_out = smem;
    }
  }
  *b_out = b;
  return best >= 0.0;
}

// ------------------------------------------------------------------ launchers

static int grid_for(fp_ctx ctx, uint64_t ntiles, int per_sm) {
  uint64_t g = (uint64_t)ctx->num_sms * per_sm;
  if (ntiles < g) g = ntiles;
  return (int)(g ? g : 1);
}

// Full tiles of 4096 words through k_pack_small (32-bit words, k in 2..5, p < 128, aligned);
// returns the number of words done.
static uint64_t pack_small(fp_ctx ctx, const fp_dqt_params& prm, const uint8_t* coeffs, uint32_t* words,
                           uint64_t count, cudaStream_t st) {
  const uint64_t ntiles = count / 4096;
  if (ntiles == 0 || prm.p >= 128 || prm.k < 2 || prm.k > 5 || ((((uintptr_t)coeffs) | ((uintptr_t)words)) & 15u))
    return 0;
  const size_t smem = 2 * 4096 * (prm.k + 4) + 64;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 4);
#define FP_PACK_K(KK)                                                                                          \
  case KK:                                                                                                     \
    cudaFuncSetAttribute(k_pack_small<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
    FP_LAUNCH(ctx, "k_pack_small", st, (k_pack_small<KK><<<grid, 256, smem, st>>>(coeffs, words, ntiles, prm.b, \
                                                                                    prm.p, ctx->d_err)));       \
    break;
  switch (prm.k) {
    FP_PACK_K(2)
    FP_PACK_K(3)
    FP_PACK_K(4)
    FP_PACK_K(5)
  }
#undef FP_PACK_K
  return ntiles * 4096;
}

// Full tiles of 4096 words through k_unpack_small (32-bit words, ndig in {3, 5, 7}, a lane-table
// correction mode, aligned); returns the number of words done.
static uint64_t unpack_small(fp_ctx ctx, const RedqParams& P, const uint32_t* words, uint8_t* coeffs,
                             uint64_t count, cudaStream_t st) {
  const uint64_t ntiles = count / 4096;
  const uint32_t nd = P.ndig;
  if (ntiles == 0 || (nd != 3 && nd != 5 && nd != 7) ||
      (P.mode != CORR_NONE && P.mode != CORR_SHFL3 && P.mode != CORR_SHFL2) ||
      ((((uintptr_t)coeffs) | ((uintptr_t)words)) & 15u))
    return 0;
  const size_t smem = 2 * 4096 * (4 + nd) + 64;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 4);
#define FP_UNPACK_K(ND, MODE)                                                                                    \
  if (nd == ND && P.mode == MODE) {                                                                              \
    cudaFuncSetAttribute(k_unpack_small<ND, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    FP_LAUNCH(ctx, "k_unpack_small", st,                                                                         \
              (k_unpack_small<ND, MODE><<<grid, 256, smem, st>>>(words, coeffs, ntiles, P, ctx->d_err)));        \
  }
  FP_UNPACK_K(3, CORR_NONE) FP_UNPACK_K(3, CORR_SHFL3) FP_UNPACK_K(3, CORR_SHFL2)
  FP_UNPACK_K(5, CORR_NONE) FP_UNPACK_K(5, CORR_SHFL3) FP_UNPACK_K(5, CORR_SHFL2)
  FP_UNPACK_K(7, CORR_NONE) FP_UNPACK_K(7, CORR_SHFL3) FP_UNPACK_K(7, CORR_SHFL2)
#undef FP_UNPACK_K
  return ntiles * 4096;
}

template <typename W>
static fp_status pack_t(fp_ctx ctx, const fp_dqt_params& prm, const uint8_t* coeffs, void* words,
                        size_t count, cudaStream_t st) {
  if (prm.qform == FP_Q_P_POW2) {
    const size_t smem_q = TILE * prm.k;
    const int grid_q = grid_for(ctx, (count + TILE - 1) / TILE, 8);
    FP_LAUNCH(ctx, "k_pack_pq", st,
              k_pack_pq<W><<<grid_q, TILE, smem_q, st>>>(coeffs, (W*)words, count, prm.k, (uint64_t)prm.p << prm.b,
                                                         prm.p, ctx->d_err));
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  if (std::is_same<W, uint32_t>::value) {
    const uint64_t done = pack_small(ctx, prm, coeffs, (uint32_t*)words, count, st);
    FP_CUDA(cudaGetLastError());
    coeffs += done * prm.k;
    words = (W*)words + done;
    count -= done;
    if (count == 0) return FP_OK;
  }
  size_t smem = TILE * prm.k;
  int grid = grid_for(ctx, (count + TILE - 1) / TILE, 8);
  FP_LAUNCH(ctx, "k_pack", st, k_pack<W><<<grid, TILE, smem, st>>>(coeffs, (W*)words, count, prm.k, prm.b, prm.p, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

fp_status launch_pack(fp_ctx ctx, const fp_dqt_params& prm, const uint8_t* coeffs, void* words,
                      size_t count, cudaStream_t st) {
  switch (prm.word) {
    case FP_WORD_F64: return pack_t<double>(ctx, prm, coeffs, words, count, st);
    case FP_WORD_F32: return pack_t<float>(ctx, prm, coeffs, words, count, st);
    case FP_WORD_U64: return pack_t<uint64_t>(ctx, prm, coeffs, words, count, st);
    default: return pack_t<uint32_t>(ctx, prm, coeffs, words, count, st);
  }
}

template <typename W>
static fp_status unpack_t(fp_ctx ctx, const fp_dqt_params& prm, const void* words, uint8_t* coeffs,
                          size_t count, cudaStream_t st) {
  RedqParams P = make_redq(prm.p, prm.b, prm.ndig);
  if (prm.qform == FP_Q_P_POW2) {
    const size_t smem = TILE * prm.ndig;
    const int grid = grid_for(ctx, (count + TILE - 1) / TILE, 8);
    FP_LAUNCH(ctx, "k_unpack_pq", st,
              k_unpack_pq<W><<<grid, TILE, smem, st>>>((const W*)words, coeffs, count, P, prm.b));
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  if (std::is_same<W, uint32_t>::value) {
    const uint64_t done = unpack_small(ctx, P, (const uint32_t*)words, coeffs, count, st);
    FP_CUDA(cudaGetLastError());
    words = (const W*)words + done;
    coeffs += done * prm.ndig;
    count -= done;
    if (count == 0) return FP_OK;
  }
  size_t smem = TILE * prm.ndig;
  int grid = grid_for(ctx, (count + TILE - 1) / TILE, 8);
  FP_LAUNCH(ctx, "k_unpack", st, k_unpack<W><<<grid, TILE, smem, st>>>((const W*)words, coeffs, count, P));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

fp_status launch_unpack(fp_ctx ctx, const fp_dqt_params& prm, const void* words, uint8_t* coeffs,
                        size_t count, cudaStream_t st) {
  switch (prm.word) {
    case FP_WORD_F64: return unpack_t<double>(ctx, prm, words, coeffs, count, st);
    case FP_WORD_F32: return unpack_t<float>(ctx, prm, words, coeffs, count, st);
    case FP_WORD_U64: return unpack_t<uint64_t>(ctx, prm, words, coeffs, count, st);
    default: return unpack_t<uint32_t>(ctx, prm, words, coeffs, count, st);
  }
}

// Exact largest packed product of a (ka coefficients) by b (kb coefficients) at q = 2^bq:
// digit j holds at most min(j+1, ka, kb, ka+kb-1-j) products of (p-1)^2.
static bool product_fits(uint32_t p, uint32_t ka, uint32_t kb, uint32_t bq, int beta) {
  uint32_t kc = ka + kb - 1;
  unsigned __int128 tot = 0, lim = (unsigned __int128)1 << beta;
  for (uint32_t j = 0; j < kc; ++j) {
    uint32_t t = j + 1;
    t = t < ka ? t : ka;
    t = t < kb ? t : kb;
    t = t < kc - j ? t : kc - j;
    if ((uint64_t)j * bq >= 100) return false;
    tot += ((unsigned __int128)t * (p - 1) * (p - 1)) << (j * bq);
    if (tot >= lim) return false;
  }
  return true;
}

// q for a single-word product: smallest 2^b above the largest digit min(ka, kb) (p-1)^2
// (Eq. bounds with n = 1, strict); b >= 1 and q >= p.
static uint32_t poly_qbits(uint32_t p, uint32_t ka, uint32_t kb) {
  uint64_t D = (uint64_t)(ka < kb ? ka : kb) * (p - 1) * (p - 1);
  uint32_t b = 1;
  while ((1ull << b) <= D || (1ull << b) < p) ++b;
  return b;
}

template <typename W>
static fp_status polymul_word_t(fp_ctx ctx, uint32_t p, const uint8_t* A, uint32_t ka, const uint8_t* B,
                                uint32_t kb, uint8_t* C, size_t batch, uint32_t bq, cudaStream_t st) {
  uint32_t kc = ka + kb - 1;
  RedqParams P = make_redq(p, bq, kc);
  // full tiles of 2048 pairs on the bulk-copy path when the arrays are 16-byte aligned and a
  // tile pair of buffers fits comfortably in shared memory; the rest on the per-thread path
  if (std::is_same<W, uint32_t>::value) {
    const uint64_t done = polymul_small(ctx, A, ka, B, kb, C, batch, P, st);
    FP_CUDA(cudaGetLastError());
    A += done * ka;
    B += done * kb;
    C += done * kc;
    batch -= done;
    if (batch == 0) return FP_OK;
  }
  constexpr uint64_t ITEMS = 256 * PolymulWordOp<W>::IPT;
  const bool aligned = ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 15u) == 0;
  const size_t tile_bytes = ITEMS * (ka + kb + kc);
  const uint64_t ntiles = batch / ITEMS;
  if (aligned && ntiles > 0 && 2 * tile_bytes <= 96 * 1024) {
    const size_t smem_b = 2 * tile_bytes + 64;
    FP_CUDA(cudaFuncSetAttribute(k_polymul_word_bulk<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    const int grid_b = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 2);
    FP_LAUNCH(ctx, "k_polymul_word_bulk", st,
              k_polymul_word_bulk<W><<<grid_b, 256, smem_b, st>>>(A, B, C, ntiles, ka, kb, P, ctx->d_err));
    FP_CUDA(cudaGetLastError());
    const uint64_t done = ntiles * ITEMS;
    A += done * ka;
    B += done * kb;
    C += done * kc;
    batch -= done;
    if (batch == 0) return FP_OK;
  }
  size_t smem = ((TILE * ka + 15) & ~15u) + ((TILE * kb + 15) & ~15u) + TILE * kc;
  int grid = grid_for(ctx, (batch + TILE - 1) / TILE, 8);
  FP_LAUNCH(ctx, "k_polymul_word", st, k_polymul_word<W><<<grid, TILE, smem, st>>>(A, B, C, batch, ka, kb, P, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

// The representation a polynomial product runs in (host only; launch_polymul follows it):
// plain; one word per operand (the first word type, in AUTO's order, whose largest product
// fits: Eq. bounds with the exact largest value); the blocked FQT; or its Karatsuba version.
// Errors: FP_EBOUND when a forced word cannot hold the product or no block size fits 64 bits.
fp_status polymul_plan(uint32_t p, uint32_t ka, uint32_t kb, int algo, fp_polymul_plan_t* pl, KaraShape* ks,
                       size_t* kara_smem) {
  const uint32_t kc = ka + kb - 1;
  *pl = fp_polymul_plan_t{};
  if (algo == FP_ALGO_PLAIN) {
    pl->kernel = FP_PM_PLAIN;
    return FP_OK;
  }
  if (algo == FP_ALGO_KARATSUBA) {
    KaraShape S;
    uint32_t bk = 0;
    size_t smem = 0;
    FP_CHECK(kara_params(p, ka, kb, &S, &bk, &smem), FP_EBOUND,
             "polymul: no Karatsuba FQT shape fits (p=%u, %u x %u coefficients)", p, ka, kb);
    pl->kernel = FP_PM_KARATSUBA;
    pl->word = FP_WORD_U64;
    pl->blk_a = pl->blk_b = S.d1;
    pl->b = bk;
    pl->ndig = 2 * S.d1 - 1;
    pl->L = S.L;
    pl->m = S.m;
    if (ks) *ks = S;
    if (kara_smem) *kara_smem = smem;
    return FP_OK;
  }
  const uint32_t bq = poly_qbits(p, ka, kb);
  // word order for AUTO: integer words first (no FP64 pipe, which is slow on this part)
  static const int order_auto[4] = {FP_WORD_U32, FP_WORD_F32, FP_WORD_U64, FP_WORD_F64};
  int forced = -1;
  if (algo == FP_ALGO_DQT_F64) forced = FP_WORD_F64;
  if (algo == FP_ALGO_DQT_U64) forced = FP_WORD_U64;
  if (algo == FP_ALGO_DQT_F32) forced = FP_WORD_F32;
  if (algo == FP_ALGO_DQT_U32) forced = FP_WORD_U32;
  if (kc <= 64) {
    for (int oi = 0; oi < 4; ++oi) {
      const int w = forced >= 0 ? forced : order_auto[oi];
      if (product_fits(p, ka, kb, bq, word_beta(w))) {
        pl->kernel = FP_PM_SINGLE_WORD;
        pl->word = (uint32_t)w;
        pl->blk_a = ka;
        pl->blk_b = kb;
        pl->b = bq;
        pl->ndig = kc;
        return FP_OK;
      }
      if (forced >= 0) break;
    }
  }
  // Blocked FQT in u64 words (Sec. 5.2): largest block size d+1 whose accumulated output word
  // fits 64 bits; digit bound: min(#blocks) (d+1) (p-1)^2 < q.
  if (forced == FP_WORD_F64 || forced == FP_WORD_F32 || forced == FP_WORD_U32) {
    set_error("polymul: %u x %u coefficients do not fit one word of the forced type; use DQT_U64 or AUTO",
              ka, kb);
    return FP_EBOUND;
  }
  uint32_t best_d1 = 0, best_b = 0;
  fqt_params(p, ka, kb, &best_d1, &best_b);
  FP_CHECK(best_d1 >= 1, FP_EBOUND, "polymul: no FQT block size fits a 64-bit word (p=%u)", p);
  pl->kernel = FP_PM_FQT;
  pl->word = FP_WORD_U64;
  pl->blk_a = pl->blk_b = best_d1;
  pl->b = best_b;
  pl->ndig = 2 * best_d1 - 1;
  return FP_OK;
}

fp_status launch_polymul(fp_ctx ctx, uint32_t p, const uint8_t* A, uint32_t da, const uint8_t* B,
                         uint32_t db, uint8_t* C, size_t batch, int algo, cudaStream_t st) {
  const uint32_t ka = da + 1, kb = db + 1, kc = ka + kb - 1;
  fp_polymul_plan_t pl;
  KaraShape S;
  size_t ksmem = 0;
  const fp_status ps = polymul_plan(p, ka, kb, algo, &pl, &S, &ksmem);
  if (ps != FP_OK) return ps;
  if (pl.kernel == FP_PM_PLAIN) {
    DivP dv = make_divp(p);
    if (kc <= 64) {
      size_t smem = ((TILE * ka + 15) & ~15u) + ((TILE * kb + 15) & ~15u) + TILE * kc;
      int grid = grid_for(ctx, (batch + TILE - 1) / TILE, 8);
      FP_LAUNCH(ctx, "k_polymul_plain_small", st, k_polymul_plain_small<<<grid, TILE, smem, st>>>(A, B, C, batch, ka, kb, p, dv, ctx->d_err));
    } else {
      int grid = grid_for(ctx, batch, 16);
      FP_LAUNCH(ctx, "k_polymul_plain_big", st, k_polymul_plain_big<<<grid, 256, 0, st>>>(A, B, C, batch, ka, kb, p, dv, ctx->d_err));
    }
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  if (pl.kernel == FP_PM_KARATSUBA) {
    RedqParams P = make_redq(p, pl.b, pl.ndig);
    FP_CUDA(cudaFuncSetAttribute(k_polymul_kara, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksmem));
    // one thread per leaf-product work item in whole warps, 128 to 256 threads (larger blocks
    // cost registers and blocks per SM and ran slower on 1023 x 1023 products)
    const uint32_t items = S.T * (((2 * S.m + 2) / 4 + 1) / 2);
    const int threads = (int)std::min<uint32_t>(256u, std::max<uint32_t>(128u, (items + 31u) & ~31u));
    int per_sm = 0;
    FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_polymul_kara, threads, ksmem));
    FP_CHECK(per_sm >= 1, FP_EUNSUPPORTED, "polymul: Karatsuba block of %d threads does not fit an SM", threads);
    const int grid = grid_for(ctx, batch, per_sm);
    FP_LAUNCH(ctx, "k_polymul_kara", st,
              k_polymul_kara<<<grid, threads, ksmem, st>>>(A, B, C, batch, ka, kb, S, P, ctx->d_err));
    FP_CUDA(cudaGetLastError());
    return FP_OK;
  }
  if (pl.kernel == FP_PM_SINGLE_WORD) {
    switch (pl.word) {
      case FP_WORD_F64: return polymul_word_t<double>(ctx, p, A, ka, B, kb, C, batch, pl.b, st);
      case FP_WORD_F32: return polymul_word_t<float>(ctx, p, A, ka, B, kb, C, batch, pl.b, st);
      case FP_WORD_U64: return polymul_word_t<uint64_t>(ctx, p, A, ka, B, kb, C, batch, pl.b, st);
      default: return polymul_word_t<uint32_t>(ctx, p, A, ka, B, kb, C, batch, pl.b, st);
    }
  }
  RedqParams P = make_redq(p, pl.b, pl.ndig);
  int grid = grid_for(ctx, batch, 16);
  FP_LAUNCH(ctx, "k_polymul_fqt", st, k_polymul_fqt<<<grid, 256, 0, st>>>(A, B, C, batch, ka, kb, pl.blk_a, P, ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

}  // namespace fpd

extern "C" fp_status fp_polymul_plan(uint32_t p, uint32_t dega, uint32_t degb, int algo, fp_polymul_plan_t* out) {
  using namespace fpd;
  FP_CHECK(out != nullptr, FP_EINVAL, "fp_polymul_plan: out is NULL");
  FP_CHECK(p >= 2 && p <= 251 && is_prime(p), FP_EINVAL, "p=%u not a prime <= 251", p);
  FP_CHECK(dega <= 1023 && degb <= 1023, FP_EINVAL, "degrees must be <= 1023");
  FP_CHECK(algo >= FP_ALGO_AUTO && algo <= FP_ALGO_KARATSUBA, FP_EINVAL, "bad algo %d", algo);
  return polymul_plan(p, dega + 1, degb + 1, algo, out, nullptr, nullptr);
}
