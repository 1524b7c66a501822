// Uneven batches of modular matrix products and dot products.
//
// Large products whose sums stay exact in fp32 go to the tensor-core kernels (p <= 17: e4m3,
// 17 < p <= 127: bf16; see "tensor-core share" below).  Everything else runs in ONE persistent
// launch of k_batch: the host planner cuts every matmul instance into 64 x 64 output tiles (64 x 64 packed words
// when the instance is packed), lists dot instances as single items, sorts the items by
// their inner dimension (longest first) and uploads the list; persistent CTAs (a multiple of
// the SM count) take items from an atomic counter until the list is exhausted -- no waiting,
// so no item can stall another.
//
// Each matmul tile runs on the warp-level tensor cores (mma.sync m16n8k16, fp32
// accumulation).  The u8 residues are converted to 16-bit while they are staged into shared
// memory (one pass over HBM), so no separate conversion kernel runs:
//   plain   bf16 residues; every chunk of the inner dimension whose sums could reach 2^24
//           is folded into a 32-bit integer accumulator (delayed reduction, Sec. 2.2);
//   packed  (p <= 3) right compression (Sec. 7.4): two centred residues of B per fp16 operand
//           at Q = 2^10, one MMA column for two columns of C; every 448 inner steps the chunk
//           word d0 + 2^10 d1 is moved into a 32-bit word D0 + 2^16 D1, and REDQ_2 (Algorithm
//           2) recovers both residues at the end.
// The packing degree (1 or 2) per (p, inner-dimension class) is chosen by a measured
// autotuner cached in the context.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <vector>

#include "fpdqt_internal.cuh"

namespace fpd {

static constexpr int BT_M = 64, BT_N = 64, BT_K = 32, BT_THREADS = 128;
static constexpr int BT_CHUNK_STEPS = 14;  // 14 x 32 = 448 inner steps per packed chunk

__device__ __forceinline__ uint32_t bsu32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int offA(int r, int c) { return r * 64 + ((c ^ ((r >> 1) & 3)) << 4); }
__device__ __forceinline__ int offB(int kr, int c) { return kr * 128 + ((c ^ (kr & 7)) << 4); }

__device__ __forceinline__ uint16_t h16(float x, bool fp16) {
  return fp16 ? __half_as_ushort(__float2half_rn(x)) : __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float centred(uint32_t v, uint32_t p) { return (p == 3 && v == 2) ? -1.0f : (float)v; }

// Load 16 consecutive bytes of a row with bounds (zeros past `limit`) as four words: one
// 16-byte load when aligned, else the aligned 4-byte words that hold them, joined by funnel
// shifts.  A word is read only if it holds a byte of the row (so no read leaves the row's
// allocation); bytes past the limit are masked off.
__device__ __forceinline__ void load16w(const uint8_t* row, int c0, int limit, uint32_t (&w)[4]) {
  const uint8_t* src = row + c0;
  const int nb = limit - c0;                 // bytes of the row from c0 on
  if (nb >= 16 && ((((uintptr_t)src) & 15u) == 0)) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(src));
    w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
    return;
  }
  if (nb <= 0) {
    w[0] = w[1] = w[2] = w[3] = 0u;
    return;
  }
  const uint32_t off = (uint32_t)((uintptr_t)src & 3u);
  const uint32_t* base = reinterpret_cast<const uint32_t*>(src - off);
  const int span = (int)off + (nb < 16 ? nb : 16);   // bytes from base that belong to the row
  uint32_t v[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = 4 * j < span ? __ldg(base + j) : 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = off ? __funnelshift_r(v[j], v[j + 1], 8 * off) : v[j];
  if (nb < 16) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int keep = nb - 4 * j;            // valid bytes in word j
      w[j] = keep >= 4 ? w[j] : (keep <= 0 ? 0u : (w[j] & ((1u << (8 * keep)) - 1u)));
    }
  }
}

// bf16 bits of two residue bytes (bytes s0, s1 of w, values <= 255): the float 2^23 + v has v in
// its low mantissa bits, so subtracting 2^23 gives float(v) exactly; its top 16 bits are the bf16.
__device__ __forceinline__ uint32_t bf16x2_of_bytes(uint32_t w, uint32_t s0, uint32_t s1) {
  const float f0 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650u + s0)) - 8388608.0f;
  const float f1 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650u + s1)) - 8388608.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632u);
}

__device__ void run_dot(const BInst& I, uint32_t* err) {
  __shared__ uint64_t red[BT_THREADS / 32];
  uint64_t acc = 0;
  uint32_t bad = 0;
  uint32_t done = 0;
  if (((((uintptr_t)I.A) | ((uintptr_t)I.B)) & 15u) == 0) {
    // 16 residues of each operand per load; four 4-way byte products (dp4a) per load pair, each
    // at most 4 (p-1)^2 < 2^18, summed in 32 bits per load pair and in 64 bits across them
    const uint32_t nv = I.k / 16, pp4 = 0x01010101u * I.p;
    const uint4* va = reinterpret_cast<const uint4*>(I.A);
    const uint4* vb = reinterpret_cast<const uint4*>(I.B);
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
      const uint4 x = __ldg(va + i), y = __ldg(vb + i);
      bad |= __vcmpgeu4(x.x, pp4) | __vcmpgeu4(x.y, pp4) | __vcmpgeu4(x.z, pp4) | __vcmpgeu4(x.w, pp4) |
             __vcmpgeu4(y.x, pp4) | __vcmpgeu4(y.y, pp4) | __vcmpgeu4(y.z, pp4) | __vcmpgeu4(y.w, pp4);
      acc += __dp4a(x.x, y.x, __dp4a(x.y, y.y, __dp4a(x.z, y.z, __dp4a(x.w, y.w, 0u))));
    }
    done = nv * 16;
  }
  for (uint32_t i = done + threadIdx.x; i < I.k; i += blockDim.x) {
    uint32_t a = I.A[i], b = I.B[i];
    bad |= (a >= I.p) | (b >= I.p);
    acc += a * b;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < BT_THREADS / 32; ++w) t += red[w];
    *reinterpret_cast<uint32_t*>(I.C) = (uint32_t)(t % I.p);
  }
  if (bad) flag_error(err, ERR_RANGE);
  __syncthreads();
}

__device__ void run_tile(const BInst& I, int tm, int tn, uint8_t* smem, uint32_t* err) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = tm * BT_M, w0 = tn * BT_N;  // first row, first output word
  const bool packed = I.packed != 0;
  const uint32_t p = I.p;
  uint8_t* sA = smem;                 // [2][64 x 32] 16-bit, 4 KB each
  uint8_t* sB = smem + 2 * 4096;      // [2][32 x 64] 16-bit, 4 KB each
  __shared__ uint8_t ptab_b[1024];
  fill_pair_table(ptab_b, I.P);
  Corrector corr;
  corr.init(I.P, ptab_b);

  float acc[2][4][4];
  uint32_t R[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) { acc[i][j][q] = 0.f; R[i][j][q] = 0u; }

  const int ksteps = (int)((I.k + BT_K - 1) / BT_K);
  const int chunk_steps = packed ? BT_CHUNK_STEPS : (int)I.plain_chunk_steps;
  uint32_t bad = 0;
  // staging registers: residue bytes as words (byte j of the 16 at byte j % 4 of word j / 4)
  uint32_t ra[4], rb[8];
  const int a_row = tid >> 1, a_h = tid & 1;
  const int b_kr = tid >> 2, b_q = tid & 3;
  const uint32_t pp4 = 0x01010101u * p;
  auto gload = [&](int ks) {
    const int kb = ks * BT_K;
    const int r = m0 + a_row;
    if (r < (int)I.m) {
      load16w(I.A + (size_t)r * I.k, kb + 16 * a_h, (int)I.k, ra);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) ra[j] = 0u;
    }
    const int kr = kb + b_kr;
    uint32_t t0[4] = {0u, 0u, 0u, 0u}, t1[4] = {0u, 0u, 0u, 0u};
    if (kr < (int)I.k) {
      const uint8_t* brow = I.B + (size_t)kr * I.n;
      if (packed) {
        load16w(brow, 2 * w0 + 32 * b_q, (int)I.n, t0);
        load16w(brow, 2 * w0 + 32 * b_q + 16, (int)I.n, t1);
      } else {
        load16w(brow, w0 + 16 * b_q, (int)I.n, t0);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) { rb[j] = t0[j]; rb[4 + j] = t1[j]; }
  };
  auto sstore = [&](int buf) {
    uint32_t o[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bad |= __vcmpgeu4(ra[q], pp4);          // zero bytes past a row's end pass the check
      if (packed) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t b0 = (ra[q] >> (16 * h)) & 0xFFu, b1 = (ra[q] >> (16 * h + 8)) & 0xFFu;
          o[2 * q + h] = (uint32_t)h16(centred(b0, p), true) | ((uint32_t)h16(centred(b1, p), true) << 16);
        }
      } else {
        o[2 * q] = bf16x2_of_bytes(ra[q], 0, 1);
        o[2 * q + 1] = bf16x2_of_bytes(ra[q], 2, 3);
      }
    }
    uint8_t* a = sA + buf * 4096;
    *reinterpret_cast<uint4*>(a + offA(a_row, 2 * a_h)) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(a + offA(a_row, 2 * a_h + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
    if (packed) {
      // word j: c(byte 2j) + 2^10 c(byte 2j + 1) of the 32 bytes
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        bad |= __vcmpgeu4(rb[q], pp4);
        const uint32_t x = rb[q];
        const float x0 = centred(x & 0xFFu, p) + 1024.0f * centred((x >> 8) & 0xFFu, p);
        const float x1 = centred((x >> 16) & 0xFFu, p) + 1024.0f * centred(x >> 24, p);
        o[q] = (uint32_t)h16(x0, true) | ((uint32_t)h16(x1, true) << 16);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bad |= __vcmpgeu4(rb[q], pp4);
        o[2 * q] = bf16x2_of_bytes(rb[q], 0, 1);
        o[2 * q + 1] = bf16x2_of_bytes(rb[q], 2, 3);
      }
    }
    uint8_t* b = sB + buf * 4096;
    *reinterpret_cast<uint4*>(b + offB(b_kr, 2 * b_q)) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(b + offB(b_kr, 2 * b_q + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
  };
  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (packed) {
            const int32_t y = __float_as_int(acc[i][j][q] + 12582912.0f);   // 0x4B400000 + word
            const int32_t d1 = (y - (0x4B400000 - 512)) >> 10;
            R[i][j][q] += (uint32_t)(y - 0x4B400000) + (uint32_t)(d1 * (65536 - 1024));
          } else {
            R[i][j][q] += __float2uint_rn(acc[i][j][q]);
          }
          acc[i][j][q] = 0.f;
        }
  };

  __syncthreads();  // previous item finished with the shared buffers
  gload(0);
  sstore(0);
  __syncthreads();
  int in_chunk = 0;
  const uint32_t idesc_dummy = 0;
  (void)idesc_dummy;
  for (int ks = 0; ks < ksteps; ++ks) {
    const int buf = ks & 1;
    if (ks + 1 < ksteps) gload(ks + 1);
    const uint8_t* a = sA + buf * 4096;
    const uint8_t* b = sB + buf * 4096;
#pragma unroll
    for (int k16 = 0; k16 < 2; ++k16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + (lane & 15);
        const int c = 2 * k16 + (lane >> 4);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(af[i][0]), "=r"(af[i][1]), "=r"(af[i][2]), "=r"(af[i][3])
                     : "r"(bsu32(a + offA(r, c))));
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int kr = 16 * k16 + (lane & 7) + (((lane >> 3) & 1) << 3);
        const int c = 4 * wn + 2 * jj + (lane >> 4);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(bfr[2 * jj][0]), "=r"(bfr[2 * jj][1]), "=r"(bfr[2 * jj + 1][0]), "=r"(bfr[2 * jj + 1][1])
                     : "r"(bsu32(b + offB(kr, c))));
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (packed)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
          else
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
        }
    }
    if (++in_chunk == chunk_steps) {
      fold();
      in_chunk = 0;
    }
    if (ks + 1 < ksteps) sstore(buf ^ 1);
    __syncthreads();
  }
  if (in_chunk) fold();
  if (bad) flag_error(err, ERR_RANGE);
  // epilogue: words -> residues (REDQ_2 for packed words, mod p for plain sums)
  const int g = lane >> 2, t = lane & 3;
  const uint32_t koff = I.k;                 // offset making centred digit sums non-negative
  const uint32_t offp = koff % p;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + wm * 32 + i * 16 + g + ((q >> 1) << 3);
        const int wc = w0 + wn * 32 + j * 8 + 2 * t + (q & 1);
        const bool own = row < (int)I.m && wc < (int)I.nw;
        if (packed) {
          uint32_t mu0, mu1;
          redq2_u32(R[i][j][q] + koff * 65537u, I.P, corr, mu0, mu1);
          uint32_t r0 = mu0 + p - offp, r1 = mu1 + p - offp;
          r0 = r0 >= p ? r0 - p : r0;
          r1 = r1 >= p ? r1 - p : r1;
          if (own) {
            uint8_t* dst = I.C + (size_t)row * I.n + 2 * wc;
            dst[0] = (uint8_t)r0;
            if (2 * wc + 1 < (int)I.n) dst[1] = (uint8_t)r1;
          }
        } else if (own) {
          I.C[(size_t)row * I.n + wc] = (uint8_t)modp32(R[i][j][q], I.P.dv, p);
        }
      }
}

__global__ void __launch_bounds__(BT_THREADS, 4) k_batch(const BInst* __restrict__ insts, const BItem* __restrict__ items,
                                                      uint32_t nitems, uint32_t* counter, uint32_t* err) {
  __shared__ __align__(128) uint8_t smem[4 * 4096];
  __shared__ uint32_t s_item;
  __shared__ BInst s_inst;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= nitems) break;
    const BItem item = items[it];
    if (threadIdx.x == 0) s_inst = insts[item.inst];
    __syncthreads();
    const BInst I = s_inst;
    if (I.kind == 1) run_dot(I, err);
    else run_tile(I, item.tm, item.tn, smem, err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host planning

static uint32_t kclass(uint32_t k) {
  uint32_t c = 0;
  while ((1u << c) < k) ++c;
  return c;
}

// Packed (two residues per word) or plain for this (p, k class): measured once per class.
static bool choose_packed(fp_ctx ctx, uint32_t p, uint32_t k, cudaStream_t st);

// The checks batch_prepare applies to instance i (returns FP_OK or the error, message set).
fp_status batch_check(const fp_instance& x, size_t i) {
  FP_CHECK(x.kind <= 1, FP_EINVAL, "fp_batch_run: instance %zu has kind %u", i, x.kind);
  FP_CHECK(x.p >= 2 && x.p <= 251 && is_prime(x.p), FP_EINVAL, "fp_batch_run: instance %zu p=%u", i, x.p);
  FP_CHECK(x.A && x.B && x.C, FP_EINVAL, "fp_batch_run: instance %zu has a null pointer", i);
  if (x.kind == 1) {
    FP_CHECK(x.k >= 1, FP_EINVAL, "fp_batch_run: dot instance %zu has length 0", i);
    return FP_OK;
  }
  FP_CHECK(x.m >= 1 && x.n >= 1 && x.k >= 1 && x.m <= 65535u * BT_M && x.n <= 65535u * BT_N, FP_EINVAL,
           "fp_batch_run: instance %zu sizes m=%u n=%u k=%u", i, x.m, x.n, x.k);
  FP_CHECK((uint64_t)x.k * (x.p - 1) * (x.p - 1) < (1ull << 32), FP_EBOUND,
           "fp_batch_run: instance %zu k (p-1)^2 >= 2^32", i);
  return FP_OK;
}

fp_status batch_prepare(fp_ctx ctx, const fp_instance* in, size_t count, cudaStream_t st, bool measure_only,
                        std::vector<BInst>& insts, std::vector<BItem>& items) {
  insts.assign(count, BInst{});
  items.clear();
  items.reserve(count * 4);
  for (size_t i = 0; i < count; ++i) {
    const fp_instance& x = in[i];
    fp_status cs = batch_check(x, i);
    if (cs != FP_OK) return cs;
    BInst b{};
    b.A = x.A; b.B = x.B; b.C = x.C; b.kind = x.kind; b.p = x.p;
    const uint64_t pp = (uint64_t)(x.p - 1) * (x.p - 1);
    if (x.kind == 1) {
      b.m = b.n = 1; b.k = x.k;
      b.P = make_redq(x.p, 16, 1);
      insts[i] = b;
      items.push_back(BItem{(uint32_t)i, 0, 0});
      continue;
    }
    b.m = x.m; b.n = x.n; b.k = x.k;
    b.packed = (!measure_only && x.p <= 3 && x.k <= 32767 && choose_packed(ctx, x.p, x.k, st)) ? 1u : 0u;
    if (measure_only) b.packed = x.reserved ? 1u : 0u;  // the autotuner's probe sets it explicitly
    b.nw = b.packed ? (x.n + 1) / 2 : x.n;
    // plain: fold before the fp32 sums can reach 2^24
    uint64_t steps = pp ? ((1ull << 24) - 1) / (pp * BT_K) : 1u << 20;
    b.plain_chunk_steps = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(steps, 1u << 20));
    b.P = b.packed ? make_redq(x.p, 16, 2) : make_redq(x.p, 16, 1);
    insts[i] = b;
    const uint32_t tmn = (x.m + BT_M - 1) / BT_M, tnn = (b.nw + BT_N - 1) / BT_N;
    for (uint32_t tm = 0; tm < tmn; ++tm)
      for (uint32_t tn = 0; tn < tnn; ++tn) items.push_back(BItem{(uint32_t)i, (uint16_t)tm, (uint16_t)tn});
  }
  // longest inner dimension first (largest items first keeps the persistent CTAs balanced)
  std::stable_sort(items.begin(), items.end(),
                   [&](const BItem& a, const BItem& b) { return insts[a.inst].k > insts[b.inst].k; });
  return FP_OK;
}

size_t batch_plan_bytes(size_t ninst, size_t nitems) {
  return ((ninst * sizeof(BInst) + 255) & ~(size_t)255) + ((nitems * sizeof(BItem) + 255) & ~(size_t)255) + 256;
}

// Lay the plan out in host staging memory `h` (batch_plan_bytes long) in the device layout.
void batch_plan_write(const std::vector<BInst>& insts, const std::vector<BItem>& items, uint8_t* h) {
  const size_t ib = (insts.size() * sizeof(BInst) + 255) & ~(size_t)255;
  memcpy(h, insts.data(), insts.size() * sizeof(BInst));
  memcpy(h + ib, items.data(), items.size() * sizeof(BItem));
  memset(h + ib + ((items.size() * sizeof(BItem) + 255) & ~(size_t)255), 0, 256);  // counter
}

// Launch the persistent kernel on a plan already resident at `d` (same layout).
fp_status batch_launch_plan(fp_ctx ctx, size_t ninst, size_t nitems, uint8_t* d, cudaStream_t st) {
  const size_t ib = (ninst * sizeof(BInst) + 255) & ~(size_t)255;
  const size_t tb = (nitems * sizeof(BItem) + 255) & ~(size_t)255;
  const int grid = (int)std::min<size_t>(nitems, (size_t)ctx->num_sms * 8);
  FP_LAUNCH(ctx, "k_batch", st,
            k_batch<<<grid, BT_THREADS, 0, st>>>((const BInst*)d, (const BItem*)(d + ib), (uint32_t)nitems,
                                                 (uint32_t*)(d + ib + tb), ctx->d_err));
  FP_CUDA(cudaGetLastError());
  return FP_OK;
}

static fp_status plan_and_launch(fp_ctx ctx, const fp_instance* in, size_t count, cudaStream_t st,
                                 bool measure_only) {
  std::vector<BInst> insts;
  std::vector<BItem> items;
  fp_status s = batch_prepare(ctx, in, count, st, measure_only, insts, items);
  if (s != FP_OK) return s;
  const size_t bytes = batch_plan_bytes(insts.size(), items.size());
  s = ensure_scratch(ctx, bytes, 1, st);
  if (s != FP_OK) return s;
  std::vector<uint8_t> h(bytes);
  batch_plan_write(insts, items, h.data());
  // pageable source: cudaMemcpyAsync returns once the bytes are staged, so h may go away
  FP_CUDA(cudaMemcpyAsync(ctx->scratch2, h.data(), bytes, cudaMemcpyHostToDevice, st));
  return batch_launch_plan(ctx, insts.size(), items.size(), (uint8_t*)ctx->scratch2, st);
}

// Autotuner probe: a synthetic batch of 16 instances 256 x 256 x k (device buffers from the
// context's autotune arena), timed packed and plain; the faster choice is cached per
// (p, k class).  Runs once per class; synchronises the stream.
static __global__ void k_fill_mod(uint8_t* x, size_t n, uint32_t p, uint32_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    x[i] = (uint8_t)(h % p);
  }
}

static bool choose_packed(fp_ctx ctx, uint32_t p, uint32_t k, cudaStream_t st) {
  const uint64_t key = (0xBA7Cull << 48) | ((uint64_t)p << 16) | kclass(k);
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return it->second != 0;
  // fixed rule (packing pays once a chunk is full) with tuning off, or inside a stream capture,
  // where the probe's allocation and synchronisation are not allowed (not cached then)
  if (!ctx->autotune || stream_capturing(st)) return k >= 448;
  const uint32_t kk = 1u << kclass(k), dim = 256, nin = 16;
  const size_t per = (size_t)dim * kk;          // one A (dim x kk) or one B (kk x dim)
  const size_t cper = (size_t)dim * dim;        // one C (dim x dim)
  void* buf = nullptr;
  bool packed = k >= 448;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (timed && cudaMalloc(&buf, 2 * per * nin + cper * nin) == cudaSuccess) {
    uint8_t* A = (uint8_t*)buf;
    uint8_t* Cb = A + 2 * per * nin;
    k_fill_mod<<<ctx->num_sms * 4, 256, 0, st>>>(A, 2 * per * nin, p, 12345u + p);
    std::vector<fp_instance> v(nin);
    for (uint32_t i = 0; i < nin; ++i) {
      v[i] = fp_instance{0, p, dim, dim, kk, 0, A + per * i, A + per * (nin + i), Cb + cper * i};
    }
    float best[2] = {1e30f, 1e30f};
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep)
      for (int pk = 0; pk < 2 && ok; ++pk) {
        for (auto& x : v) x.reserved = (uint32_t)pk;
        float ms = 0;
        ok = cudaEventRecord(e0, st) == cudaSuccess &&
             plan_and_launch(ctx, v.data(), v.size(), st, true) == FP_OK &&
             cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        best[pk] = std::min(best[pk], ms);
      }
    cudaStreamSynchronize(st);
    cudaFree(buf);
    if (ok) {
      packed = best[1] < best[0];
      ctx->tune[key] = packed ? 1 : 0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();   // a failed probe leaves no sticky error for a later, unrelated check
  return packed;        // not cached when the probe failed: the fixed rule stands
}

// ---------------------------------------------------------------- tensor-core share of a batch
//
// Matrix products whose residues are exact e4m3 values as they stand (p <= 17, unsigned sums
// k (p-1)^2 < 2^23) or once centred (p <= 31: |c| <= p/2 <= 15, 2 k (p/2)^2 + p < 2^23), so
// that the sums stay below 2^23 (the range of the e4m3 epilogue's reduction, see k_tcg.cu), and
// that fill enough of their 128 x 256 x 32 blocks run on the pre-tiled tcgen05 kernel
// (k_mm_f8g_pre) instead of the mma.sync tiles of k_batch; larger p (up to 127,
// k (p-1)^2 < 2^24, m, n >= 64) on the bf16 kernel.  One launch of k_tile_pack lays every routed operand out as the 16 KB swizzled blocks that kernel's
// stages copy (layout in fpdqt_internal.cuh): residues range-checked and centred, zero outside
// the matrix, so the caller's arrays may have any row stride and alignment.  Then one
// tensor-core launch takes the whole share (up to F8_PRE_CAP products per launch).

static constexpr uint64_t BT_TC_MIN_MACS = 1ull << 21;

struct TileJob {
  const uint8_t* src;  // rows x cols residues, leading dimension ld
  uint8_t* dst;        // the job's first 16 KB block
  uint32_t rows, cols, ld, p;
  uint32_t nkt;        // k tiles of the product
  uint32_t is_b;       // 0: A, blocks (mb, kt); 1: B, blocks (nb, kt, h)
  uint32_t blk0;       // first block of the job in the launch's numbering
  uint32_t centre;     // 1: residues > p/2 become the codes of r - p (p > 17, or sums too large)
};

// The 16 bytes of a row from column col on (nvalid of them belong to the row; none when
// nvalid <= 0), zero past the row.  Only the aligned 4-byte words that hold a byte of the row are
// read (so no read leaves the row's allocation), all issued before any is used.
__device__ __forceinline__ void chunk_load(const uint8_t* rowp, int col, int nvalid, uint32_t (&w)[4]) {
  const uint8_t* s = rowp + col;
  const uint32_t off = (uint32_t)((uintptr_t)s & 3u);
  const uint32_t* b = reinterpret_cast<const uint32_t*>(s - off);
  const int span = (int)off + min(nvalid, 16);          // bytes from b that belong to the row
  uint32_t v[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = 4 * j < span ? __ldg(b + j) : 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t x = __funnelshift_r(v[j], v[j + 1], 8 * off);   // off = 0: v[j]
    const int keep = nvalid - 4 * j;                               // bytes of word j in the row
    w[j] = keep >= 4 ? x : (keep <= 0 ? 0u : x & ((1u << (8 * keep)) - 1u));
  }
}

// One CTA per contiguous range of 16 KB blocks (its first job found once by binary search, then
// advanced block by block).  Thread t writes chunks t, t + 256, t + 512, t + 768 of a block
// (coalesced): chunk o is block row o / 8 at swizzled position o % 8, i.e. source chunk
// (o % 8) ^ (row % 8) of that row.  Every byte is range-checked (r < p: r + 128 - p has bit 7
// clear) and, for centred jobs, r > p/2 becomes the e4m3 code of -(p - r) (sign bit | (p - r)).
// Block rows of A past m and sectors of B past n are not written: they only reach accumulator
// rows or columns the epilogue never stores.  The inner-dimension padding (A columns, B rows
// past k) is written as zeros: it meets every output.
__global__ void __launch_bounds__(256) k_tile_pack(const TileJob* __restrict__ jobs, uint32_t njobs, uint32_t nblocks,
                                                   uint32_t* err) {
  const uint32_t per = (nblocks + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = blockIdx.x * per, b1 = min(nblocks, b0 + per);
  if (b0 >= b1) return;
  uint32_t jb = 0, hi = njobs - 1;               // the last job whose first block is <= b0
  while (jb < hi) {
    const uint32_t mid = (jb + hi + 1) >> 1;
    if (jobs[mid].blk0 <= b0) jb = mid;
    else hi = mid - 1;
  }
  uint32_t bad = 0;
  for (uint32_t bi = b0; bi < b1; ++bi) {
    while (jb + 1 < njobs && jobs[jb + 1].blk0 <= bi) ++jb;
    const TileJob& J = jobs[jb];
    const uint32_t local = bi - J.blk0, nkt = J.nkt, is_b = J.is_b;
    uint32_t rb, cb;                            // block row (128 rows), block column (128 bytes)
    if (!is_b) {
      rb = local / nkt;
      cb = local - rb * nkt;
    } else {
      const uint32_t nb = local / (2 * nkt), rem = local - nb * 2 * nkt;
      rb = rem >> 1;
      cb = 2 * nb + (rem & 1u);
    }
    const uint8_t* src = J.src;
    const uint32_t rows = J.rows, cols = J.cols, ld = J.ld, p = J.p, centre = J.centre;
    uint4* dst = reinterpret_cast<uint4*>(J.dst + (size_t)local * F8_BLOCK);
    const uint32_t pk = 0x01010101u * (128u - p), hk = 0x01010101u * (127u - (p >> 1)), P4 = 0x01010101u * p;
    uint32_t w[4][4];
    bool st[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t o = threadIdx.x + 256u * i;
      const uint32_t r = o >> 3, c = (o & 7u) ^ (r & 7u);
      const uint32_t row = rb * 128 + r, col = cb * 128 + 16 * c;
      const bool row_in = row < rows;
      // chunks c and c ^ 1 share a 32-byte sector (at positions o % 8 and (o % 8) ^ 1): a B
      // chunk past n is still written (zeros) when its partner is not, so that no sector is
      // half written (which would cost a read-modify-write in DRAM)
      st[i] = is_b ? (cb * 128 + 16 * (c & ~1u) < cols || !row_in) : row_in;
      chunk_load(src + (size_t)(row_in ? row : 0) * ld, (int)col, row_in ? (int)cols - (int)col : -64, w[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t x = w[i][j];
        bad |= x | (x + pk);
        if (centre) {
          const uint32_t gt = (((x + hk) & 0x80808080u) >> 7) * 0xFFu;   // 0xFF where r > p/2
          w[i][j] = (gt & ((P4 - x) | 0x80808080u)) | (~gt & x);
        }
      }
      if (st[i]) dst[threadIdx.x + 256u * i] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
  }
  if (bad & 0x80808080u) flag_error(err, ERR_RANGE);
}

// 1: pre-tiled e4m3 products (p <= 31); 2: bf16 products (31 < p <= 127, residues exact in bf16
// and the conversion's range check valid); 0: the batch kernel.  The e4m3 kernel computes whole
// 128 x 256 x 32 blocks: a product goes there when those padded MACs are at least 2^21 and at
// most 32 times its own (a thin product still runs far faster there than on the mma.sync tiles
// of the batch kernel), or when k >= 128 however thin it is (the batch kernel takes k in steps
// of 32 with one step of prefetch, so a long k would make one of its items the longest part of
// the whole launch).
static bool f8_unsigned_ok(uint32_t p, uint64_t k) { return p <= 17 && k * (p - 1) * (p - 1) < (1ull << 23); }
static bool f8_centred_ok(uint32_t p, uint64_t k) { return p <= 31 && 2 * k * (p / 2) * (p / 2) + p < (1ull << 23); }

static int batch_tc_route(const fp_instance& x) {
  const bool mm = x.kind == 0 && x.A && x.B && x.C && x.p >= 2 && x.p <= 127 && is_prime(x.p) && x.k >= 1 &&
                  x.m <= (1u << 30) && x.n <= (1u << 30) && x.k <= (1u << 30);
  if (!mm) return 0;
  const unsigned __int128 macs = (unsigned __int128)((uint64_t)x.m * x.n) * x.k;
  if (f8_unsigned_ok(x.p, x.k) || f8_centred_ok(x.p, x.k)) {
    const unsigned __int128 padded = (unsigned __int128)(((x.m + 127ull) & ~127ull) * ((x.n + 255ull) & ~255ull)) *
                                     ((x.k + 31ull) & ~31ull);
    return padded >= BT_TC_MIN_MACS && (padded <= 32 * macs || x.k >= 128) ? 1 : 0;
  }
  const bool big = x.m >= 64 && x.n >= 64 && macs >= BT_TC_MIN_MACS;
  return big && (uint64_t)x.k * (x.p - 1) * (x.p - 1) < (1ull << 24) ? 2 : 0;
}

// The tensor-core share: e4m3 products (pack in one launch, then one pre-tiled launch per
// F8_PRE_CAP products) and bf16 products (conversion in one launch, grouped k_mm_t16 launches),
// from one scratch allocation.  Lock held.
static fp_status batch_run_tc(fp_ctx ctx, const std::vector<const fp_instance*>& tc,
                              const std::vector<const fp_instance*>& t16, cudaStream_t st) {
  auto up256 = [](uint64_t x) { return (x + 255) & ~(uint64_t)255; };
  // longest inner dimension first: the persistent schedule starts the longest tiles earliest
  std::vector<const fp_instance*> v(tc);
  std::stable_sort(v.begin(), v.end(), [](const fp_instance* a, const fp_instance* b) { return a->k > b->k; });
  const size_t np = v.size();
  // scratch: [problems | first tiles | pack jobs] (one upload) | operand blocks | bf16 share
  const uint64_t o_tile0 = up256(np * sizeof(F8PreProb));
  const uint64_t o_jobs = o_tile0 + up256(np * sizeof(int));
  const uint64_t desc = o_jobs + up256(2 * np * sizeof(TileJob));
  const uint64_t o_blocks = (desc + 1023) & ~(uint64_t)1023;
  std::vector<uint8_t> h(desc);
  F8PreProb* prob = reinterpret_cast<F8PreProb*>(h.data());
  int* tile0 = reinterpret_cast<int*>(h.data() + o_tile0);
  TileJob* jobs = reinterpret_cast<TileJob*>(h.data() + o_jobs);
  std::vector<int> chunk_tiles;                 // tiles of each launch of F8_PRE_CAP problems
  uint64_t nblk = 0;
  int tiles = 0;
  for (size_t i = 0; i < np; ++i) {
    const fp_instance& x = *v[i];
    if (i % F8_PRE_CAP == 0) {
      if (i) chunk_tiles.push_back(tiles);
      tiles = 0;
    }
    const uint32_t kt = (x.k + 127) / 128, tm = (x.m + 127) / 128, tn = (x.n + 255) / 256;
    const uint64_t a_blk = nblk, b_blk = a_blk + (uint64_t)tm * kt;
    nblk = b_blk + (uint64_t)tn * kt * 2;
    // residues as they stand (codes 0..16) while the unsigned sums stay below 2^23, else centred
    const uint32_t centre = f8_unsigned_ok(x.p, x.k) ? 0u : 1u;
    jobs[2 * i] = TileJob{x.A, (uint8_t*)(uintptr_t)a_blk, x.m, x.k, x.k, x.p, kt, 0u, (uint32_t)a_blk, centre};
    jobs[2 * i + 1] = TileJob{x.B, (uint8_t*)(uintptr_t)b_blk, x.k, x.n, x.n, x.p, kt, 1u, (uint32_t)b_blk, centre};
    const uint64_t hh = x.p / 2, bound = (uint64_t)x.k * hh * hh;
    const uint64_t pt = centre ? (bound + x.p - 1) / x.p * x.p : 0;   // p T >= k (p/2)^2
    F8PreProb& q = prob[i];
    q.At = (const uint8_t*)(uintptr_t)a_blk;
    q.Bt = (const uint8_t*)(uintptr_t)b_blk;
    q.C = x.C;
    q.m = (int)x.m;
    q.n = (int)x.n;
    q.ldc = (int)x.n;
    q.ktiles = (int)kt;
    q.klast = (int)((x.k - 128 * (kt - 1) + 31) / 32);
    q.tn = (int)tn;
    q.p = x.p;
    q.off18 = (float)pt / 262144.0f;                   // exact: p T < 2^23
    tile0[i] = tiles;
    tiles += (int)(tm * tn);
  }
  if (np) chunk_tiles.push_back(tiles);
  FP_CHECK(nblk < (1ull << 32), FP_EINVAL, "fp_batch_run: tensor-core share too large for one call");
  std::vector<fp_mm_problem> prob16(t16.size());
  std::vector<const fp_mm_problem*> ptr16(t16.size());
  for (size_t i = 0; i < t16.size(); ++i) {
    const fp_instance& x = *t16[i];
    prob16[i] = fp_mm_problem{x.p, (int)x.m, (int)x.n, (int)x.k, x.A, (int)x.k, x.B, (int)x.n, x.C, (int)x.n};
    ptr16[i] = &prob16[i];
  }
  const uint64_t f8_end = o_blocks + nblk * F8_BLOCK;
  const uint64_t off16 = (f8_end + 1023) & ~(uint64_t)1023;
  const uint64_t total = t16.empty() ? f8_end : off16 + t16_batch_bytes(ptr16.data(), ptr16.size());
  {
    fp_status s = ensure_scratch(ctx, total + 1024, 0, st);
    if (s != FP_OK) return s;
  }
  uint8_t* base = (uint8_t*)ctx->scratch;
  if (np) {
    uint8_t* blocks = base + o_blocks;
    for (size_t i = 0; i < np; ++i) {   // block indices -> device addresses
      prob[i].At = blocks + (uintptr_t)prob[i].At * F8_BLOCK;
      prob[i].Bt = blocks + (uintptr_t)prob[i].Bt * F8_BLOCK;
      jobs[2 * i].dst = blocks + (uintptr_t)jobs[2 * i].dst * F8_BLOCK;
      jobs[2 * i + 1].dst = blocks + (uintptr_t)jobs[2 * i + 1].dst * F8_BLOCK;
    }
    fp_status s = upload_staged(ctx, 0, base, h.data(), desc, st);
    if (s != FP_OK) return s;
    const uint32_t njobs = (uint32_t)(2 * np);
    // one wave of resident CTAs: each takes a fixed contiguous range of blocks, so a CTA that
    // had to wait for a free slot would finish a whole range after the others
    static int per_sm = 0;
    if (per_sm == 0) FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_pack, 256, 0));
    const int grid = (int)std::min<uint64_t>(nblk, (uint64_t)ctx->num_sms * std::max(1, per_sm));
    FP_LAUNCH(ctx, "k_tile_pack", st,
              k_tile_pack<<<grid, 256, 0, st>>>((const TileJob*)(base + o_jobs), njobs, (uint32_t)nblk, ctx->d_err));
    FP_CUDA(cudaGetLastError());
    for (size_t c = 0; c < chunk_tiles.size(); ++c) {
      const size_t i0 = c * F8_PRE_CAP, cnt = std::min<size_t>(F8_PRE_CAP, np - i0);
      s = launch_mm_f8_pretiled(ctx, (const F8PreProb*)base + i0, (const int*)(base + o_tile0) + i0, (int)cnt,
                                chunk_tiles[c], st);
      if (s != FP_OK) return s;
    }
  }
  if (t16.empty()) return FP_OK;
  return launch_mm_t16_plain_batch(ctx, ptr16.data(), ptr16.size(), base + off16, st);
}

}  // namespace fpd

extern "C" fp_status fp_batch_run(fp_ctx ctx, const fp_instance* instances, size_t count, void* stream) {
  using namespace fpd;
  FP_CHECK(ctx != nullptr, FP_EINVAL, "fp_batch_run: ctx is NULL");
  if (count == 0) return FP_OK;
  FP_CHECK(instances != nullptr, FP_EINVAL, "fp_batch_run: instances is NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = as_stream(stream);
  std::vector<const fp_instance*> tc, t16;
  std::vector<fp_instance> rest;
  rest.reserve(count);
  // every instance checked before anything is enqueued (the routed ones satisfy the checks by
  // construction); the batch kernel's plan is built while the GPU runs the tensor-core share
  for (size_t i = 0; i < count; ++i) {
    const int route = batch_tc_route(instances[i]);
    if (route == 1) {
      tc.push_back(&instances[i]);
    } else if (route == 2) {
      t16.push_back(&instances[i]);
    } else {
      fp_status s = batch_check(instances[i], i);
      if (s != FP_OK) return s;
      rest.push_back(instances[i]);
    }
  }
  if (!tc.empty() || !t16.empty()) {
    fp_status s = batch_run_tc(ctx, tc, t16, st);
    if (s != FP_OK) return s;
  }
  if (rest.empty()) return FP_OK;
  std::vector<BInst> insts;
  std::vector<BItem> items;
  {
    fp_status s = batch_prepare(ctx, rest.data(), rest.size(), st, false, insts, items);
    if (s != FP_OK) return s;
  }
  const size_t bytes = batch_plan_bytes(insts.size(), items.size());
  fp_status s = ensure_scratch(ctx, bytes, 1, st);
  if (s != FP_OK) return s;
  std::vector<uint8_t> h(bytes);
  batch_plan_write(insts, items, h.data());
  s = upload_staged(ctx, 1, ctx->scratch2, h.data(), bytes, st);
  if (s != FP_OK) return s;
  return batch_launch_plan(ctx, insts.size(), items.size(), (uint8_t*)ctx->scratch2, st);
}
