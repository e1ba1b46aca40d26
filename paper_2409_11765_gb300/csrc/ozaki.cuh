// ozaki.cuh -- FP64-accurate matrix products on the BF16 tensor cores, by
// error-free splitting of the operands into digit planes (the scheme of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012).
//
// GB300 issues FP64 at 1/64 of its FP32 rate and about 1/1500 of its dense
// BF16 tensor rate, so the eigensolver's long FP64 products (the Gram matrix
// V^T V of the orthogonalisation, the blocked back-transformation) run here.
//
// Digits. Row r of an operand (R rows by K, K-major) with exponent e_r
// (|x_rk| < 2^e_r for every k) is rounded once to the fixed-point integer
//   F_rk = round(x_rk 2^(8S - 2 - e_r)),   |F_rk| <= 2^(8S-2),
// and F is cut into S balanced base-256 digits d_1..d_S in [-128, 127]
// (d_1 most significant), so that
//   x_rk = 2^(e_r + 2) sum_p d_p 2^(-8p)   (to within 2^(e_r - 8S + 1)).
// Every digit is an integer of at most 8 significant bits, exact in BF16.
//
// Products. Plane pair (p, q) contributes d^A_p d^B_q 2^(eA + eB + 4 - 8(p+q));
// pairs with p + q <= S + 1 are kept (the rest weigh below 2^-8(S+2) of the
// leading term). Bucket t = p + q gathers the t - 1 pairs of equal weight in
// its own TMEM accumulator: their integer products are below 2^14, and over a
// K chunk of 128 the bucket sums stay below 7 * 2^21 < 2^24, so the FP32
// accumulation of the tensor core is exact. After every chunk the buckets are
// drained: the five heaviest into one 64-bit fixed-point integer per output
// element (exact), the two lightest (below 2^-40 of the leading term) into an
// FP32 sum; the epilogue forms the FP64 value once, (W + L) 2^(eA + eB - 44).
// Besides the final rounding, the error is that of the representation
// (2^(e - 55) per entry) and of the neglected pairs (below
// 6 * 2^(eA + eB - 54) per term of the K sum).
//
// Packed operand layout in global memory (what the tile loads with bulk
// copies): rows padded to a multiple of 128, K to a multiple of 32; the block
// of 64 rows x 32 K of digit plane p, for row block rb and K chunk kc, is 4 KB
// at byte ((rb * nks + kc) * S + p) * 4096, in the K-major no-swizzle core
// matrix layout of the tensor core (8 rows x 8 BF16 = 128 contiguous bytes,
// core (g, c) at ((g * 4) + c) * 128).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "tc_common.cuh"

namespace cmaes_gb300 {

constexpr int kOzS = 7;                    // digits per operand (54 bits)
constexpr int kOzBM = 128;                 // output rows per tile (TMEM lanes)
constexpr int kOzBN = 64;                  // output columns per tile
constexpr int kOzKS = 32;                  // K per staged chunk
constexpr int kOzDrain = 4;                // staged chunks per exact bucket sum (K = 128)
constexpr int kOzBlk = 4096;               // bytes of one 64 x 32 digit block
constexpr int kOzStage = kOzS * 3 * kOzBlk;  // A (two blocks) + B (one block) per plane
constexpr int kOzSmem = 2 * kOzStage + 1024;
constexpr int kOzTmemCols = 512;           // kOzS buckets x 64 columns, rounded up
constexpr int kOzZeroExp = -4000;          // exponent of an all-zero row
constexpr int kOzNT = 256;

__host__ __device__ inline long long oz_pitch(int nks) {  // bytes per 64-row block
  return static_cast<long long>(nks) * kOzS * kOzBlk;
}
__host__ __device__ inline int oz_rows_padded(int R) { return (R + 127) / 128 * 128; }
__host__ __device__ inline int oz_nks(int K) { return (K + kOzKS - 1) / kOzKS; }
__host__ __device__ inline size_t oz_bytes(int R, int K) {
  return static_cast<size_t>(oz_rows_padded(R) / 64) * static_cast<size_t>(oz_pitch(oz_nks(K)));
}

// --------------------------------------------------------------------------
// Digit extraction
// --------------------------------------------------------------------------
// Exponent E with |x| < 2^E (frexp's), kOzZeroExp for zero and subnormals.
__device__ __forceinline__ int oz_exponent(double x) {
  const int be = static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF);
  return be == 0 ? kOzZeroExp : be - 1022;
}

// BF16 bit pattern of an integer d in [-128, 127] (exact: at most 8
// significant bits, so the low half of the FP32 pattern is zero).
__device__ __forceinline__ uint32_t oz_bf16_bits(int d) {
  const float f = __int_as_float(0x4B000000 | (d + 128)) - 8388736.0f;
  return __float_as_uint(f) >> 16;
}

// The kOzS digits of x for a row with exponent e, as BF16 patterns
// (out[0] = d_1, the most significant).
__device__ __forceinline__ void oz_digits(double x, int e, uint32_t (&out)[kOzS]) {
  const long long bits = __double_as_longlong(x);
  const int be = static_cast<int>((bits >> 52) & 0x7FF);
  long long F = 0;
  if (be != 0 && e > kOzZeroExp) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = be - 1077 + 8 * kOzS - e;  // <= 8S - 55 since |x| < 2^e
    if (sh >= 0) F = mant << sh;
    else if (sh > -63) F = (mant + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) F = -F;
  }
#pragma unroll
  for (int p = kOzS - 1; p >= 0; --p) {
    const int d = static_cast<int>(static_cast<signed char>(F & 0xFF));
    F = (F - d) >> 8;
    out[p] = oz_bf16_bits(d);
  }
}

// Byte offset of digit (row r, k) inside a 64 x 32 block.
__device__ __forceinline__ int oz_off(int r, int k) {
  return (((r >> 3) * 4 + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// --------------------------------------------------------------------------
// Packing of one 64-row block of an operand: x(r, k) = get(r, k) for r < R,
// k < K (zero elsewhere; get is called only inside), rows rb * 64 ..
// rb * 64 + 63, K chunks 0 .. nks - 1. kfast: consecutive k are contiguous in
// memory (then 4 threads read 32 consecutive k of a row), else consecutive
// rows are (a warp reads 32 consecutive rows). All kOzNT threads of the block
// call it; sh_e holds 64 ints. Writes the row exponents to e_out[r] (r < the
// padded row count).
// --------------------------------------------------------------------------
template <class Get>
__device__ __forceinline__ void oz_pack_block_get(const Get& get, bool kfast, int R, int K, int rb, int nks,
                                                  unsigned char* __restrict__ out, int* __restrict__ e_out,
                                                  int* sh_e) {
  const int tid = threadIdx.x;
  const int rl = kfast ? (tid >> 2) : (tid & 63);
  const int oc = kfast ? (tid & 3) : (tid >> 6);
  const int r = rb * 64 + rl;
  if (tid < 64) sh_e[tid] = kOzZeroExp;
  __syncthreads();
  int emax = kOzZeroExp;
  if (r < R) {
    for (int k = oc * 8; k < K; k += 32) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k + u < K) emax = max(emax, oz_exponent(get(r, k + u)));
    }
  }
  atomicMax(&sh_e[rl], emax);
  __syncthreads();
  const int e = sh_e[rl];
  if (oc == 0) e_out[r] = e;
  unsigned char* base = out + static_cast<long long>(rb) * oz_pitch(nks);
  for (int kc = 0; kc < nks; ++kc) {
    uint32_t pk[kOzS][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const int k = kc * kOzKS + oc * 8 + u;
      const double x0 = (r < R && k < K) ? get(r, k) : 0.0;
      const double x1 = (r < R && k + 1 < K) ? get(r, k + 1) : 0.0;
      uint32_t d0[kOzS], d1[kOzS];
      oz_digits(x0, e, d0);
      oz_digits(x1, e, d1);
#pragma unroll
      for (int p = 0; p < kOzS; ++p) pk[p][u >> 1] = d0[p] | (d1[p] << 16);
    }
    unsigned char* blk = base + static_cast<long long>(kc) * kOzS * kOzBlk + oz_off(rl, oc * 8);
#pragma unroll
    for (int p = 0; p < kOzS; ++p)
      *reinterpret_cast<uint4*>(blk + p * kOzBlk) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
  }
}

// The same for a strided view x(r, k) = src[r * sr + k * sk].
__device__ __forceinline__ void oz_pack_block(const double* __restrict__ src, long long sr, long long sk, int R,
                                              int K, int rb, int nks, unsigned char* __restrict__ out,
                                              int* __restrict__ e_out, int* sh_e) {
  oz_pack_block_get(
      [=] __device__(int r, int k) { return src[static_cast<long long>(r) * sr + static_cast<long long>(k) * sk]; },
      sk == 1, R, K, rb, nks, out, e_out, sh_e);
}

// 2^e as a double (0 or infinity outside the normal range).
__device__ __forceinline__ double oz_pow2(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
  return ldexp(1.0, e);
}

// x 2^e as a double for an integer x, assembled on the bit pattern (the
// leading bit found by clz, rounded to nearest even above 2^53): the same
// value as double(x) * 2^e without FP64 arithmetic. Outside the normal range
// it falls back to the FP64 operations.
__device__ __forceinline__ double oz_i2d_scaled(long long x, int e) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = static_cast<unsigned long long>(x) & 0x8000000000000000ull;
  unsigned long long m = x < 0 ? 0ull - static_cast<unsigned long long>(x) : static_cast<unsigned long long>(x);
  const int msb = 63 - __clzll(static_cast<long long>(m));
  int ex = msb + e;
  if (msb > 52) {
    const int sh = msb - 52;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    m >>= sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m >> 53) {
        m >>= 1;
        ++ex;
      }
    }
  } else {
    m <<= (52 - msb);
  }
  if (ex < -1022 || ex > 1023) return static_cast<double>(x) * oz_pow2(e);
  return __longlong_as_double(static_cast<long long>(sgn | (static_cast<unsigned long long>(ex + 1023) << 52) |
                                                     (m & 0xFFFFFFFFFFFFFull)));
}

// f 2^e as a double for a float f, on the bit pattern (exact; zero for a
// zero or subnormal f), the FP64 operations outside the normal range.
__device__ __forceinline__ double oz_f2d_scaled(float f, int e) {
  const unsigned u = __float_as_uint(f);
  const int fe = static_cast<int>((u >> 23) & 0xFF);
  if (fe == 0) return 0.0;
  const int ex = fe - 127 + e;
  if (ex < -1022 || ex > 1023) return static_cast<double>(f) * oz_pow2(e);
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(u >> 31) << 63) |
                                                     (static_cast<unsigned long long>(ex + 1023) << 52) |
                                                     (static_cast<unsigned long long>(u & 0x7FFFFFu) << 29)));
}

// The FP64 value of an output element from its tile sums (oz_tile) and the
// exponents of its row of A and its row of B: (W + L) 2^(eA + eB - 44), both
// terms scaled exactly, one FP64 addition.
__device__ __forceinline__ double oz_value(long long W, float L, int ea, int eb) {
  if (ea <= kOzZeroExp || eb <= kOzZeroExp) return 0.0;
  const int e = ea + eb - 44;
  return oz_i2d_scaled(W, e) + oz_f2d_scaled(L, e);
}

// --------------------------------------------------------------------------
// Bulk copies and transaction-counted mbarriers
// --------------------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  float a[16], b[16];
  tmem_ld16(taddr, a);
  tmem_ld16(taddr + 16, b);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    v[q] = a[q];
    v[16 + q] = b[q];
  }
}


// --------------------------------------------------------------------------
// The tile: out(i, j) for rows i0 + 0..127 of A and columns j0 + 0..63 (rows
// of B), K = nks * 32. Shared state set up by oz_begin. Each thread ends with
// row i0 + 32 (warp & 3) + lane, columns j0 + 32 (warp >> 2) + 0..31 as
// W + L in units of 2^(eA + eB - 44): W the exact sum of the five heaviest
// buckets, L the two lightest (FP32, weight below 2^-40 of the leading
// term). Returns false (uniformly) if a wait ran out.
// --------------------------------------------------------------------------
struct OzCtx {
  unsigned char* base;  // 1024-aligned dynamic shared memory (two stages)
  uint64_t* bar;        // full[2], empty[2], drain
  uint32_t tmem;
  int uses[2];          // completed uses of each stage buffer (phase bookkeeping)
  int drains;           // completed drains
};

__device__ __forceinline__ void oz_begin(OzCtx& cx, unsigned char* dyn, uint64_t* bar5, uint32_t* tmem_slot) {
  cx.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~static_cast<uintptr_t>(1023));
  cx.bar = bar5;
  cx.uses[0] = cx.uses[1] = 0;
  cx.drains = 0;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tmem_slot)), "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(&bar5[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cx.tmem = *tmem_slot;
}

__device__ __forceinline__ void oz_end(OzCtx& cx) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(cx.tmem), "r"(kOzTmemCols));
}

__device__ __forceinline__ bool oz_tile(OzCtx& cx, const unsigned char* __restrict__ A, long long a_pitch, int a_rb,
                        const unsigned char* __restrict__ B, long long b_pitch, int b_rb, int nks,
                        long long (&W)[32], float (&L)[32]) {
  const int tid = threadIdx.x, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    W[q] = 0;
    L[q] = 0.0f;
  }
  if (nks <= 0) return true;
  const unsigned char* a0 = A + static_cast<long long>(a_rb) * a_pitch;
  const unsigned char* a1 = a0 + a_pitch;
  const unsigned char* b0 = B + static_cast<long long>(b_rb) * b_pitch;
  uint64_t* full = cx.bar;
  uint64_t* empty = cx.bar + 2;
  uint64_t* drain = cx.bar + 4;
  const uint32_t idesc = tc_idesc<1>(kOzBN);
  __shared__ int sh_fail;
  if (tid == 0) sh_fail = 0;
  auto issue = [&](int c) {
    const int b = c & 1;
    unsigned char* sa = cx.base + b * kOzStage;
    unsigned char* sb = sa + kOzS * 2 * kOzBlk;
    mbar_expect_tx(&full[b], kOzStage);
    const long long ko = static_cast<long long>(c) * kOzS * kOzBlk;
#pragma unroll 1
    for (int p = 0; p < kOzS; ++p) {
      bulk_g2s(sa + p * 2 * kOzBlk, a0 + ko + p * kOzBlk, kOzBlk, &full[b]);
      bulk_g2s(sa + p * 2 * kOzBlk + kOzBlk, a1 + ko + p * kOzBlk, kOzBlk, &full[b]);
      bulk_g2s(sb + p * kOzBlk, b0 + ko + p * kOzBlk, kOzBlk, &full[b]);
    }
  };
  const int ndrain = (nks + kOzDrain - 1) / kOzDrain;
  bool ok = true;
  for (int dc = 0; dc < ndrain; ++dc) {
    if (tid == 0 && ok) {
      if (dc == 0) {
        // buffer 0 may still be read by MMAs of an earlier tile of this CTA
        if (cx.uses[0] > 0 && !mbar_wait_bounded(&empty[0], (cx.uses[0] - 1) & 1)) ok = false;
        if (ok) issue(0);
      }
      const int c1 = min(nks, (dc + 1) * kOzDrain);
      for (int c = dc * kOzDrain; c < c1 && ok; ++c) {
        const int b = c & 1;
        // the data of chunk c has landed (use number uses[b] of this buffer)
        if (!mbar_wait_bounded(&full[b], cx.uses[b] & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned char* sa = cx.base + b * kOzStage;
        const unsigned char* sb = sa + kOzS * 2 * kOzBlk;
        const bool first = (c == dc * kOzDrain);
#pragma unroll 1
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll 1
          for (int p = 0; p < kOzS; ++p) {
            const uint64_t da = tc_sdesc(smem_u32(sa + p * 2 * kOzBlk) + ks * 256, 128, 512);
#pragma unroll 1
            for (int q = 0; q + p < kOzS; ++q) {
              const uint64_t db = tc_sdesc(smem_u32(sb + q * kOzBlk) + ks * 256, 128, 512);
              const uint32_t acc = (first && ks == 0 && p == 0) ? 0u : 1u;
              tc_mma<1>(cx.tmem + static_cast<uint32_t>((p + q) * kOzBN), da, db, idesc, acc);
            }
          }
        }
        tc_commit(&empty[b]);
        ++cx.uses[b];
        // refill the other buffer once the MMAs of chunk c - 1 are done; they
        // run while the MMAs of chunk c wait in the queue behind them
        if (c + 1 < nks) {
          const int nb = (c + 1) & 1;
          if (cx.uses[nb] > 0 && !mbar_wait_bounded(&empty[nb], (cx.uses[nb] - 1) & 1)) {
            ok = false;
            break;
          }
          issue(c + 1);
        }
      }
      if (ok) tc_commit(drain);
      if (!ok) sh_fail = 1;
    }
    __syncthreads();
    if (sh_fail) {
      ok = false;
      break;
    }
    // every thread: wait for this chunk's bucket sums, then drain them
    const bool got = mbar_wait_bounded(drain, cx.drains & 1);
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    ++cx.drains;
    tc_fence_after();
    const uint32_t taddr = cx.tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 32 * (warp >> 2);
    // the five heaviest buckets as one 64-bit fixed-point integer (exact), the
    // lighter ones in FP32 in units of the fifth
#pragma unroll 1
    for (int t = 0; t < 5; ++t) {
      float v[32];
      tmem_ld32(taddr + t * kOzBN, v);
      const int sh = 32 - 8 * t;
#pragma unroll
      for (int q = 0; q < 32; ++q) W[q] += static_cast<long long>(__float2int_rn(v[q])) << sh;
    }
#pragma unroll 1
    for (int t = 5; t < kOzS; ++t) {
      float v[32];
      tmem_ld32(taddr + t * kOzBN, v);
      const float w = __int_as_float((127 - 8 * (t - 4)) << 23);  // 2^(-8(t-4))
#pragma unroll
      for (int q = 0; q < 32; ++q) L[q] = __fmaf_rn(v[q], w, L[q]);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (!ok && tid == 0) {
    // let issued copies land and issued MMAs finish before the shared memory
    // and TMEM are released (each wait is bounded)
    for (int b = 0; b < 2; ++b) {
      mbar_wait_bounded(&full[b], cx.uses[b] & 1);
      if (cx.uses[b] > 0) mbar_wait_bounded(&empty[b], (cx.uses[b] - 1) & 1);
    }
  }
  return ok;
}

}  // namespace cmaes_gb300
