// tc_common.cuh -- 5th-generation tensor-core (tcgen05) building blocks for
// the mixed-precision GEMMs: shared-memory matrix descriptors, the instruction
// descriptor, TMEM allocation and loads, MMA issue/commit and a bounded
// mbarrier wait, plus a double-buffered 128 x N tile driver.
//
// Operand layout in shared memory: K-major, no swizzle. A tile of R rows by
// KC elements is a grid of "core matrices" of 8 rows x 16 bytes (4 TF32 or 8
// BF16 values), each stored as 128 contiguous bytes; core (row group g, k
// group c) sits at byte ((g * kcores) + c) * 128 with kcores = KC * esz / 16.
// One MMA consumes 32 bytes of K (8 TF32 / 16 BF16 values): two core matrices
// along K (leading-dimension offset 128 bytes), row groups 8 rows apart
// (stride-dimension offset kcores * 128 bytes).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cmaes_gb300 {

constexpr int kTcKC = 32;              // K elements staged per chunk
constexpr long long kTcWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
  return d;                              // base offset 0, no swizzle
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128.
// KIND 0: kind::tf32 (A, B TF32); KIND 1: kind::f16 with BF16 A, B.
template <int KIND>
__device__ __forceinline__ uint32_t tc_idesc(int N) {
  const uint32_t fmt = KIND == 0 ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(128 >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == 0)
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
  return ok != 0;
}

// Waits for the given phase with a time limit; returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity)) {
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Rounding to the tensor-core input formats (round to nearest).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int KIND>
struct TcElem;
template <>
struct TcElem<0> {
  using T = float;
  static constexpr int esz = 4;
  __device__ static T from(float x) { return to_tf32(x); }
  __device__ static float back(T x) { return x; }
};
template <>
struct TcElem<1> {
  using T = __nv_bfloat16;
  static constexpr int esz = 2;
  __device__ static T from(float x) { return __float2bfloat16_rn(x); }
  __device__ static float back(T x) { return __bfloat162float(x); }
};

// Byte offset of element (r, k) inside a staged chunk with kcores core
// matrices along K.
template <int KIND>
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  constexpr int esz = TcElem<KIND>::esz;
  constexpr int kcores = kTcKC * esz / 16;
  return static_cast<uint32_t>(((r >> 3) * kcores + ((k * esz) >> 4)) * 128 + (r & 7) * 16 + ((k * esz) & 15));
}

// Split a float into hi + lo in the input format; x - hi is exact in FP32, so
// hi + lo carries 22 (TF32) or 16 (BF16) significant bits of x.
template <int KIND>
__device__ __forceinline__ void tc_split32(float x, typename TcElem<KIND>::T& hi, typename TcElem<KIND>::T& lo) {
  hi = TcElem<KIND>::from(x);
  lo = TcElem<KIND>::from(x - TcElem<KIND>::back(hi));
}

// Split x into hi + lo in the input format (hi = round(x), lo = round(x - hi)).
template <int KIND>
__device__ __forceinline__ void tc_split(double x, typename TcElem<KIND>::T& hi, typename TcElem<KIND>::T& lo) {
  hi = TcElem<KIND>::from(static_cast<float>(x));
  lo = TcElem<KIND>::from(static_cast<float>(x - static_cast<double>(TcElem<KIND>::back(hi))));
}

// Shared-memory plan of the tile driver: two buffers, each holding A (128
// rows) and B (up to 256 rows), hi and (with SPLIT) lo parts.
template <int KIND, bool SPLIT>
struct TcPlan {
  static constexpr int esz = TcElem<KIND>::esz;
  static constexpr int a_bytes = 128 * kTcKC * esz;
  static constexpr int b_bytes = 256 * kTcKC * esz;
  static constexpr int parts = SPLIT ? 2 : 1;
  static constexpr int buf_bytes = parts * (a_bytes + b_bytes);
  static constexpr int bytes = 2 * buf_bytes + 1024;  // + alignment slack
};

struct TcCtx {
  unsigned char* base;  // 1024-aligned dynamic shared memory
  uint64_t* mbar;       // two mbarriers (one per buffer)
  uint32_t tmem;        // accumulator base (256 columns)
  int chunk;            // chunks issued so far (phase bookkeeping)
  int failed;
};

// One 128 x N x K product accumulated in TMEM columns [0, N). stage(buf, k0,
// a_hi, a_lo, b_hi, b_lo) fills chunk [k0, k0 + kTcKC) of both operands (all
// threads); zero beyond the valid rows / K must be written by the stager.
// Thread 0 issues the MMAs; with SPLIT the product is hi*hi + hi*lo + lo*hi.
// Returns false (uniformly) if a wait timed out.
template <int KIND, bool SPLIT, class Stage>
__device__ bool tc_tile(TcCtx& ctx, int N, int K, const Stage& stage) {
  using P = TcPlan<KIND, SPLIT>;
  const int nch = (K + kTcKC - 1) / kTcKC;
  const uint32_t idesc = tc_idesc<KIND>(N);
  constexpr int kcores = kTcKC * P::esz / 16;
  constexpr int mmas = kTcKC * P::esz / 32;
  int failed = 0;
  for (int c = 0; c < nch; ++c) {
    const int g = ctx.chunk + c;  // global chunk index on this CTA
    const int buf = g & 1;
    unsigned char* bb = ctx.base + buf * P::buf_bytes;
    unsigned char* a_hi = bb;
    unsigned char* b_hi = bb + P::a_bytes;
    unsigned char* a_lo = SPLIT ? bb + P::a_bytes + P::b_bytes : nullptr;
    unsigned char* b_lo = SPLIT ? a_lo + P::a_bytes : nullptr;
    if (g >= 2) {
      // the MMAs that last read this buffer must be complete
      int ok = 1;
      if (threadIdx.x == 0) ok = mbar_wait_bounded(&ctx.mbar[buf], ((g - 2) >> 1) & 1);
      failed |= __syncthreads_or(!ok);
      if (failed) break;
    }
    stage(c * kTcKC, a_hi, a_lo, b_hi, b_lo);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
      for (int s = 0; s < mmas; ++s) {
        const uint32_t sbo = kcores * 128;
        const uint64_t ah = tc_sdesc(smem_u32(a_hi) + s * 256, 128, sbo);
        const uint64_t bh = tc_sdesc(smem_u32(b_hi) + s * 256, 128, sbo);
        const uint32_t first = (c == 0 && s == 0) ? 0u : 1u;
        tc_mma<KIND>(ctx.tmem, ah, bh, idesc, first);
        if (SPLIT) {
          const uint64_t al = tc_sdesc(smem_u32(a_lo) + s * 256, 128, sbo);
          const uint64_t bl = tc_sdesc(smem_u32(b_lo) + s * 256, 128, sbo);
          tc_mma<KIND>(ctx.tmem, ah, bl, idesc, 1u);
          tc_mma<KIND>(ctx.tmem, al, bh, idesc, 1u);
        }
      }
      tc_commit(&ctx.mbar[buf]);
    }
  }
  if (!failed) {
    const int g = ctx.chunk + nch - 1;
    int ok = 1;
    if (threadIdx.x == 0) ok = mbar_wait_bounded(&ctx.mbar[g & 1], (g >> 1) & 1);
    failed |= __syncthreads_or(!ok);
  }
  tc_fence_after();
  ctx.chunk += nch;
  ctx.failed |= failed;
  return !failed;
}

// Set-up and tear-down around tc_tile calls (all threads of the CTA call them).
__device__ __forceinline__ void tc_begin(TcCtx& ctx, unsigned char* dyn, uint64_t* mbar2, uint32_t* tmem_slot) {
  ctx.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~static_cast<uintptr_t>(1023));
  ctx.mbar = mbar2;
  ctx.chunk = 0;
  ctx.failed = 0;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tmem_slot)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&mbar2[0], 1);
    mbar_init(&mbar2[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  ctx.tmem = *tmem_slot;
}

__device__ __forceinline__ void tc_end(TcCtx& ctx) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(ctx.tmem), "r"(256));
}

// Before reusing TMEM for the next tile: every thread's loads are done.
__device__ __forceinline__ void tc_tile_done() {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

}  // namespace cmaes_gb300
