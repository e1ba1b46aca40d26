// device_common.cuh -- device helpers shared by the engine's kernels:
// Philox4x32-10 draws, tile lookup over uneven searches, fixed-order block
// reductions and the FP64 GEMM tile used by the sampling, objective,
// covariance and eigensolver-setup products.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "engine.h"

namespace cmaes_gb300 {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
//   c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 52-bit uniform in (0, 1) from two words: (top 52 bits + 1/2) * 2^-52, exact.
__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  const unsigned long long v = ((static_cast<unsigned long long>(a) << 32) | b) >> 12;
  return (static_cast<double>(v) + 0.5) * 0x1p-52;
}

__device__ __forceinline__ uint32_t stream_word(int search, int restart) {
  return (static_cast<uint32_t>(search) << 8) | (static_cast<uint32_t>(restart) & 255u);
}

// Box-Muller pair for coordinates (2j, 2j+1) of candidate k in generation g.
__device__ __forceinline__ void normal_pair(uint32_t j, uint32_t k, uint32_t g, uint32_t sw,
                                            uint32_t k0, uint32_t k1, double& z0, double& z1) {
  const uint4 w = philox4x32_10(make_uint4(j, k, g, sw), k0, k1);
  const double u1 = uniform52(w.x, w.y);
  const double u2 = uniform52(w.z, w.w);
  const double r = sqrt(-2.0 * log(u1));
  const double a = (2.0 * 3.141592653589793) * u2;
  double s, c;
  sincos(a, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Uniform coordinate i of the mean of descent `restart` in [lo, hi].
__device__ __forceinline__ double restart_mean_coord(int i, int search, int restart, uint32_t k0,
                                                     uint32_t k1, double lo, double hi) {
  const uint4 w = philox4x32_10(
      make_uint4(static_cast<uint32_t>(i) >> 1, 0xFFFFFFFFu, 0xFFFFFFFFu, stream_word(search, restart)),
      k0, k1);
  const double u = (i & 1) ? uniform52(w.z, w.w) : uniform52(w.x, w.y);
  return lo + (hi - lo) * u;
}

// ---------------------------------------------------------------------------
// Tile lookup: the launch covers searches [s0, s1); tile blockIdx.x maps to
// the search whose prefix range holds off[s0] + blockIdx.x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_search(const TileMap& tm, int& local) {
  const int t = tm.off[tm.s0] + static_cast<int>(blockIdx.x);
  int lo = tm.s0, hi = tm.s1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tm.off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  local = t - tm.off[lo];
  return lo;
}

// Fixed-order block reductions (the same blockDim always sums in the same
// order, so results are reproducible run to run).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) r += sh[w];
    sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = sh[0];
    for (int w = 1; w < NT / 32; ++w) r = fmax(r, sh[w]);
    sh[0] = r;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ int block_or(int v, int* sh) {
  v = __reduce_or_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int r = 0;
  for (int w = 0; w < NT / 32; ++w) r |= sh[w];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// FP64 GEMM tile: out(i, j) = sum_k a(i, k) b(k, j) over a 64 x 64 tile,
// K in steps of 16, 256 threads with 4 x 4 outputs each. The operand
// accessors are functors so that gathers (selected columns), offsets
// (x - x*) and transposes are applied while staging into shared memory;
// A_I_CONTIG / B_K_CONTIG say which index is contiguous in memory so the
// staging loads coalesce. The k-order of every sum is fixed (ascending).
// ---------------------------------------------------------------------------
constexpr int kGBM = 64, kGBN = 64, kGBK = 16, kGNT = 256;

struct GemmSmem {
  double As[kGBK][kGBM + 1];
  double Bs[kGBK][kGBN + 1];
};

template <bool A_I_CONTIG, bool B_K_CONTIG, class LA, class LB, class EPI>
__device__ __forceinline__ void gemm_tile_f64(int M, int N, int K, int i0, int j0, const LA& la,
                                              const LB& lb, const EPI& epi, GemmSmem& sm) {
  const int tid = threadIdx.x;
  const int tr = tid & 15, tc = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int k0 = 0; k0 < K; k0 += kGBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kGNT;
      int ii, kk;
      if (A_I_CONTIG) { ii = e & (kGBM - 1); kk = e >> 6; }
      else { kk = e & (kGBK - 1); ii = e >> 4; }
      const int gi = i0 + ii, gk = k0 + kk;
      sm.As[kk][ii] = (gi < M && gk < K) ? la(gi, gk) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kGNT;
      int kk, jj;
      if (B_K_CONTIG) { kk = e & (kGBK - 1); jj = e >> 4; }
      else { jj = e & (kGBN - 1); kk = e >> 6; }
      const int gk = k0 + kk, gj = j0 + jj;
      sm.Bs[kk][jj] = (gk < K && gj < N) ? lb(gk, gj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sm.As[kk][tr + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = sm.Bs[kk][tc + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + tr + 16 * r, j = j0 + tc + 16 * c;
      if (i < M && j < N) epi(i, j, acc[r][c]);
    }
}

// ---------------------------------------------------------------------------
// Plane rotation of the cyclic Jacobi method for the symmetric 2 x 2 block
// [[app, apq], [apq, aqq]] (Golub & Van Loan, Matrix Computations, §8.5):
// t = tan(phi) is the root of smaller magnitude of apq t^2 + d t - apq = 0 with
// d = aqq - app (t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), theta = d / (2 apq)),
// c = 1 / sqrt(1 + t^2), s = t c, and the rotated block is
// diag(app - t apq, aqq + t apq).
//
// GB300 runs FP64 at 1/64 of the FP32 rate and an FP64 divide or square root
// expands into a long sequence on that pipe, so t and c start from FP32 values
// and are finished in FP64 by Newton's method:
//   t: two steps on g(t) = apq t^2 + d t - apq with an FP32 reciprocal of g'(t)
//      (each step multiplies the relative error by about 2^-22);
//   c: two steps of y <- y (3 - x y^2) / 2 on x = 1 + t^2, Newton's iteration
//      for 1/y^2 = x (each step squares the relative error).
// d and apq are first scaled by a power of two (exactly) so that the larger of
// the two lies in [1, 4): the FP32 values neither overflow nor underflow.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double& t,
                                                double& c, double& s) {
  const double d = aqq - app;
  const double mx = fmax(fabs(d), fabs(apq));
  const int e = static_cast<int>((__double_as_longlong(mx) >> 52) & 0x7ff);
  const double sc = __longlong_as_double(static_cast<long long>(2046 - min(e, 2045)) << 52);
  const double ds = d * sc, as = apq * sc;
  const float df = static_cast<float>(ds), af = static_cast<float>(as);
  float tf;
  if (fabsf(af) * 0x1p40f < fabsf(df)) {
    tf = __fdividef(af, df);  // |theta| > 2^39: t = 1 / (2 theta) to FP32 precision
  } else {
    const float th = __fdividef(df, af + af);
    tf = __fdividef(th >= 0.f ? 1.f : -1.f, fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
  }
  double tt = static_cast<double>(tf);
  const double as2 = as + as;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double g = fma(fma(as, tt, ds), tt, -as);
    const double r = static_cast<double>(__fdividef(1.f, static_cast<float>(fma(as2, tt, ds))));
    tt = fma(-g, r, tt);
  }
  const double x = fma(tt, tt, 1.0), hx = 0.5 * x;
  double y = static_cast<double>(rsqrtf(static_cast<float>(x)));
#pragma unroll
  for (int it = 0; it < 2; ++it) y = fma(y, fma(-hx * y, y, 0.5), y);
  t = tt;
  c = y;
  s = tt * y;
}

// Rotation test of the cyclic Jacobi method: the pair turns when
// |apq| > tol sqrt(|app aqq|), evaluated as apq^2 > tol^2 |app aqq| (the same
// test without an FP64 square root for entries between 1e-150 and 1e150).
__device__ __forceinline__ bool jacobi_rotates(double app, double aqq, double apq, double tol2) {
  return apq != 0.0 && apq * apq > tol2 * fabs(app * aqq);
}

// The same test with an absolute floor: entries at or below `floor` never turn.
__device__ __forceinline__ bool jacobi_rotates(double app, double aqq, double apq, double tol2, double floor) {
  return fabs(apq) > floor && apq * apq > tol2 * fabs(app * aqq);
}

}  // namespace cmaes_gb300
