// kernels_gen.cu -- one CMA-ES generation over a batch of uneven searches.
//
// Paper mapping (Redon et al., "Massively parallel CMA-ES with increasing
// population"):
//   k_sample_z, k_gemm_sample   Algorithm 1 lines 4-6, Eq. (1) as one GEMM
//                               (§3.1): Z ~ N(0, I), Y = B D Z, X = m + sigma Y
//   k_gemm_objective,
//   k_colreduce_f               Algorithm 1 lines 7-9 on the built-in
//                               synthetic objectives (U = Q (X - x*), f)
//   k_rank                      the rank rk(i) behind the weights w_rk(i) of
//                               Eq. (2): ascending f, NaN as +inf, ties by index
//   k_recomb_*, k_psigma_*,
//   k_finalize                  Algorithm 1 line 10 / §2.1: mean, p_sigma,
//                               p_c and sigma updates
//   k_cov                       Eq. (2) in the rank-mu GEMM form of Eq. (3)
//   k_stop                      stop tests of §2.2 and the restart of Algorithm 2
//
// Every kernel covers a range of searches through a flattened tile list, so
// searches of different (n, lambda) share one launch; tiles beyond a search's
// current lambda exit at once, which keeps launch shapes fixed across the
// lambda changes of IPOP restarts.
#include <cmath>
#include <cuda_bf16.h>
#include "device_common.cuh"
#include "tc_common.cuh"

namespace cmaes_gb300 {

// ------------------------------- tile counts --------------------------------
int tiles_sample_z(int n, int lam_cap) { return ceil_div(ceil_div(n, 2) * lam_cap, 256); }
int tiles_gemm_panel(int n, int lam_cap) { return ceil_div(n, kGBM) * ceil_div(lam_cap, kGBN); }
int tiles_colreduce(int lam_cap) { return ceil_div(lam_cap, 8); }
int tiles_rank(int lam_cap) { return ceil_div(lam_cap, 256); }
int tiles_rank2d(int lam_cap) { return ceil_div(lam_cap, 256) * ceil_div(lam_cap, kRankChunk); }
int tiles_rows(int n) { return ceil_div(n, 256); }
int tiles_recomb(int n, int mu_cap) { return ceil_div(n, 32) * ceil_div(mu_cap, 256); }
int tiles_gemv(int n) { return ceil_div(n, 32) * ceil_div(n, 256); }
int part_doubles(int n, int ldn, int mu_cap) {
  const int a = 2 * ceil_div(mu_cap, 256), b = ceil_div(n, 256);
  return (a > b ? a : b) * ldn;
}
int tiles_sym(int n) { const int t = ceil_div(n, kGBM); return t * (t + 1) / 2; }
int tiles_square(int n) { const int t = ceil_div(n, kGBM); return t * t; }

// --------------------------- strategy parameters ----------------------------
// Tutorial defaults (Hansen, arXiv:1604.00772) for the constants the paper
// leaves to the c-cmaes code (§4.1): log weights on the best floor(lambda/2)
// points summing to one (Eq. (2)), mu_eff, c_sigma, d_sigma, c_c, c_1, c_mu,
// E||N(0,I)||, the lazy eigendecomposition period, the history length of the
// "quality not improving" test and the iteration cap.
template <int NT>
__device__ void compute_params(Search& s, const DevOptions& o, double* sh) {
  const int n = s.n, lam = s.lam, mu = lam / 2;
  const double lw = log((lam + 1) / 2.0);
  double part = 0.0;
  for (int i = threadIdx.x; i < mu; i += NT) part += lw - log(static_cast<double>(i + 1));
  const double sum = block_sum<NT>(part, sh);
  double sq = 0.0;
  for (int i = threadIdx.x; i < mu; i += NT) {
    const double wi = (lw - log(static_cast<double>(i + 1))) / sum;
    s.w[i] = wi;
    if (s.mixed) s.w32[i] = static_cast<float>(wi);
    sq += wi * wi;
  }
  const double ssq = block_sum<NT>(sq, sh);
  if (threadIdx.x == 0) {
    const double dn = static_cast<double>(n);
    const double mueff = 1.0 / ssq;
    s.mu = mu;
    s.mueff = mueff;
    s.cs = (mueff + 2.0) / (dn + mueff + 5.0);
    s.ds = 1.0 + 2.0 * fmax(0.0, sqrt((mueff - 1.0) / (dn + 1.0)) - 1.0) + s.cs;
    s.cc = (4.0 + mueff / dn) / (dn + 4.0 + 2.0 * mueff / dn);
    s.c1 = 2.0 / ((dn + 1.3) * (dn + 1.3) + mueff);
    s.cmu = fmin(1.0 - s.c1, 2.0 * (mueff - 2.0 + 1.0 / mueff) / ((dn + 2.0) * (dn + 2.0) + mueff));
    s.chin = sqrt(dn) * (1.0 - 1.0 / (4.0 * dn) + 1.0 / (21.0 * dn * dn));
    const int lazy = static_cast<int>(floor(1.0 / ((s.c1 + s.cmu) * dn * 10.0)));
    s.g_eig = o.eig_every > 0 ? o.eig_every : (lazy > 1 ? lazy : 1);
    s.hist_len = 10 + static_cast<int>(ceil(30.0 * dn / lam));
    s.max_iter = o.max_iter > 0
                     ? o.max_iter
                     : static_cast<int>(floor(100.0 + 50.0 * (dn + 3.0) * (dn + 3.0) / sqrt(static_cast<double>(lam))));
  }
  __syncthreads();
}

// Fresh descent state (Algorithm 2, "initialize"): C = B = I, D = 1, paths
// zero, sigma = sigma0. The mean is set by the caller.
template <int NT>
__device__ void reset_descent(Search& s) {
  const int n = s.n, ldn = s.ldn;
  for (int i = threadIdx.x; i < n; i += NT) {
    s.ps[i] = 0.0;
    s.pc[i] = 0.0;
    s.D[i] = 1.0;
  }
  for (long long e = threadIdx.x; e < static_cast<long long>(ldn) * n; e += NT) {
    const int i = static_cast<int>(e % ldn), j = static_cast<int>(e / ldn);
    const double v = (i == j) ? 1.0 : 0.0;
    s.C[e] = v;
    s.B[e] = v;
    s.BD[e] = v;
  }
  if (s.mixed) {  // tensor-core copy of B D: identity as well
    const int kp = s.kp;
    for (long long e = threadIdx.x; e < static_cast<long long>(n) * kp; e += NT) {
      const int i = static_cast<int>(e / kp), k = static_cast<int>(e % kp);
      const float v = (i == k) ? 1.0f : 0.0f;
      if (s.mixed == 2) static_cast<__nv_bfloat16*>(s.BDT)[e] = __float2bfloat16_rn(v);
      else static_cast<float*>(s.BDT)[e] = v;
    }
  }
  if (threadIdx.x == 0) {
    s.sigma = s.sigma0;
    s.gen = 0;
    s.hist_count = 0;
    s.eig_due = 0;
  }
}

__global__ void __launch_bounds__(256) k_init_params(Search* S, int s0, DevOptions o, int reset_state) {
  __shared__ double sh[32];
  Search& s = S[s0 + blockIdx.x];
  if (reset_state) {
    reset_descent<256>(s);
    for (int i = threadIdx.x; i < s.n; i += 256) s.best_x[i] = nan("");
    if (threadIdx.x == 0) {
      s.lam = s.lam0;
      s.restart = 0;
      s.done = 0;
      s.flags = 0;  // a restart keeps the flags that ended the previous descent
      s.best_f = INFINITY;
    }
    __syncthreads();
  }
  compute_params<256>(s, o, sh);
}

void launch_init_params(Search* S, int s0, int s1, DevOptions o, int reset_state, cudaStream_t st) {
  if (s1 > s0) k_init_params<<<s1 - s0, 256, 0, st>>>(S, s0, o, reset_state);
}

// ------------------------------- sampling -----------------------------------
// z_k ~ N(0, I): coordinates (2j, 2j+1) of candidate k come from one Philox
// call with counter (j, k, gen, search << 8 | restart).
__global__ void __launch_bounds__(256) k_sample_z(Search* S, TileMap tm, DevOptions o) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn, lam = s.lam;
  const int npairs = (n + 1) >> 1;
  const long long e = static_cast<long long>(t) * 256 + threadIdx.x;
  const int k = static_cast<int>(e / npairs), j = static_cast<int>(e % npairs);
  if (k >= lam) return;
  double z0, z1;
  if (s.mixed) {
    // the values are rounded to TF32 / BF16 right after: FP32 Box-Muller on
    // the same 52-bit uniforms (FP64 log and sincos would dominate on GB300)
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(k),
                                             static_cast<uint32_t>(s.gen), stream_word(s.index, s.restart)),
                                  o.key0, o.key1);
    const float u1 = static_cast<float>(uniform52(w.x, w.y));
    const float u2 = static_cast<float>(uniform52(w.z, w.w));
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
  } else {
    normal_pair(static_cast<uint32_t>(j), static_cast<uint32_t>(k), static_cast<uint32_t>(s.gen),
                stream_word(s.index, s.restart), o.key0, o.key1, z0, z1);
  }
  if (j == 0) s.rank[k] = 0;  // k_rank accumulates into it
  if (s.mixed) {
    // z in the tensor-core input format; the recombination reads the same values
    const long long e0 = static_cast<long long>(s.kp) * k + 2 * j;
    if (s.mixed == 2) {
      __nv_bfloat16* zc = static_cast<__nv_bfloat16*>(s.Zm);
      zc[e0] = __float2bfloat16_rn(static_cast<float>(z0));
      if (2 * j + 1 < n) zc[e0 + 1] = __float2bfloat16_rn(static_cast<float>(z1));
    } else {
      float* zc = static_cast<float*>(s.Zm);
      zc[e0] = to_tf32(static_cast<float>(z0));
      if (2 * j + 1 < n) zc[e0 + 1] = to_tf32(static_cast<float>(z1));
    }
    return;
  }
  double* col = s.Z + static_cast<long long>(ldn) * k;
  if (2 * j + 1 < n) {
    *reinterpret_cast<double2*>(col + 2 * j) = make_double2(z0, z1);
  } else {
    col[2 * j] = z0;
  }
}

void launch_sample_z(Search* S, TileMap tm, DevOptions o, cudaStream_t st) {
  if (tm.total > 0) k_sample_z<<<tm.total, 256, 0, st>>>(S, tm, o);
}

// Eq. (1) for all candidates (§3.1): Y = (B diag(D)) Z, X = m 1^T + sigma Y.
__global__ void __launch_bounds__(256) k_gemm_sample(Search* S, TileMap tm) {
  __shared__ GemmSmem sm;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn, lam = s.lam;
  const int mt = ceil_div(n, kGBM);
  const int i0 = (t % mt) * kGBM, j0 = (t / mt) * kGBN;
  if (j0 >= lam) return;
  const double* BD = s.BD;
  const double* Z = s.Z;
  double* Y = s.Y;
  double* X = s.X;
  const double* m = s.m;
  const double sigma = s.sigma;
  gemm_tile_f64<true, true>(
      n, lam, n, i0, j0,
      [=] __device__(int i, int k) { return BD[i + static_cast<long long>(ldn) * k]; },
      [=] __device__(int k, int j) { return Z[k + static_cast<long long>(ldn) * j]; },
      [=] __device__(int i, int j, double acc) {
        const long long e = i + static_cast<long long>(ldn) * j;
        Y[e] = acc;
        X[e] = m[i] + sigma * acc;
      },
      sm);
}

void launch_gemm_sample(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_gemm_sample<<<tm.total, 256, 0, st>>>(S, tm);
}

// ------------------------------- objective ----------------------------------
// Rotated objectives: U = Q (X - x*), with x - x* formed in FP64.
__global__ void __launch_bounds__(256) k_gemm_objective(Search* S, TileMap tm) {
  __shared__ GemmSmem sm;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || s.obj == 3 /* sphere: no rotation */) return;
  const int n = s.n, ldn = s.ldn, lam = s.lam;
  const int mt = ceil_div(n, kGBM);
  const int i0 = (t % mt) * kGBM, j0 = (t / mt) * kGBN;
  if (j0 >= lam) return;
  const double* Q = s.Q;
  const double* X = s.X;
  const double* xs = s.xstar;
  double* U = s.U;
  gemm_tile_f64<true, true>(
      n, lam, n, i0, j0,
      [=] __device__(int i, int k) { return Q[i + static_cast<long long>(ldn) * k]; },
      [=] __device__(int k, int j) { return X[k + static_cast<long long>(ldn) * j] - xs[k]; },
      [=] __device__(int i, int j, double acc) { U[i + static_cast<long long>(ldn) * j] = acc; },
      sm);
}

void launch_gemm_objective(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_gemm_objective<<<tm.total, 256, 0, st>>>(S, tm);
}

// f_k: one warp per candidate column, lanes stride over the rows in order and
// a fixed shuffle tree combines them.
__global__ void __launch_bounds__(256) k_colreduce_f(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || (s.mixed && s.obj != 3)) return;
  const int n = s.n, ldn = s.ldn, lam = s.lam;
  const int k = t * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= lam) return;
  double acc = 0.0;
  if (s.obj == 3) {
    const double* x = s.X + static_cast<long long>(ldn) * k;
    for (int i = lane; i < n; i += 32) {
      const double r = x[i] - s.xstar[i];
      acc += r * r;
    }
  } else if (s.obj == 1) {
    const double* u = s.U + static_cast<long long>(ldn) * k;
    for (int i = lane; i < n; i += 32) acc += s.lamdiag[i] * u[i] * u[i];
  } else {
    const double* u = s.U + static_cast<long long>(ldn) * k;
    for (int i = lane; i < n; i += 32) acc += u[i] * u[i] - 10.0 * cos((2.0 * 3.141592653589793) * u[i]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) s.f[k] = (s.obj == 2) ? 10.0 * n + acc : acc;
}

void launch_colreduce_f(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_colreduce_f<<<tm.total, 256, 0, st>>>(S, tm);
}

// --------------------------------- ranking ----------------------------------
// rank(k) = #{j : (key_j, j) < (key_k, k)} with key = f, NaN -> +inf. A
// counting rank is stable by construction; order[rank(k)] = k. The j range is
// split into chunks of kRankChunk handled by separate blocks that add their
// integer counts atomically (integer sums do not depend on the order).
// rank[] is cleared by k_sample_z (the ask/tell path also samples first).
// Order-preserving 64-bit integer key of f: NaN -> +inf, -0 -> +0, then the
// IEEE bit pattern with the sign folded so that unsigned order = numeric order.
// (Comparing integers keeps the O(lambda^2) count off GB300's slow FP64 pipe.)
__device__ __forceinline__ unsigned long long rank_key(double f) {
  if (isnan(f)) f = INFINITY;
  if (f == 0.0) f = 0.0;
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(f));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_rank(Search* S, TileMap tm) {
  __shared__ unsigned long long keys[kRankChunk];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int lam = s.lam;
  const int nkt = ceil_div(s.lam_cap, 256);
  const int kt = t % nkt, jc = t / nkt;
  const int j0 = jc * kRankChunk;
  if (kt * 256 >= lam || j0 >= lam) return;
  const int k = kt * 256 + threadIdx.x;
  const double* f = s.f;
  const int jn = min(kRankChunk, lam - j0);
  for (int q = threadIdx.x; q < jn; q += 256) keys[q] = rank_key(f[j0 + q]);
  __syncthreads();
  if (k >= lam) return;
  const unsigned long long key = rank_key(f[k]);
  int cnt = 0;
  // candidates j < k count when key_j <= key_k, candidates j > k when key_j < key_k
  const int split = min(max(k - j0, 0), jn);
  for (int jj = 0; jj < split; ++jj) cnt += keys[jj] <= key;
  for (int jj = split; jj < jn; ++jj) cnt += keys[jj] < key;
  if (cnt) atomicAdd(&s.rank[k], cnt);
}

__global__ void __launch_bounds__(256) k_order(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int k = t * 256 + threadIdx.x;
  if (k < s.lam) s.order[s.rank[k]] = k;
}

void launch_rank(Search* S, TileMap tm2d, TileMap tm, cudaStream_t st) {
  if (tm2d.total > 0) k_rank<<<tm2d.total, 256, 0, st>>>(S, tm2d);
  if (tm.total > 0) k_order<<<tm.total, 256, 0, st>>>(S, tm);
}

// ----------------------- recombination (two stages) --------------------------
// <y>_w = sum_r w_r y_{order[r]}, <z>_w likewise. Stage 1: a tile is 32 rows x
// 256 ranks; warp w sums ranks r = w, w+8, ... of the chunk, the 8 warp sums
// are added in warp order. Stage 2 adds the chunk sums in chunk order.
__global__ void __launch_bounds__(256) k_recomb_partial(Search* S, TileMap tm) {
  __shared__ double shy[8][33], shz[8][33];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn, mu = s.mu;
  const int nrt = ceil_div(n, 32);
  const int rt = t % nrt, ch = t / nrt;
  const int r0 = ch * 256;
  if (r0 >= mu) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = rt * 32 + lane;
  const int r1 = min(mu, r0 + 256);
  double ay = 0.0, az = 0.0;
  if (i < n && !s.mixed) {
    for (int r = r0 + w; r < r1; r += 8) {
      const long long col = static_cast<long long>(ldn) * s.order[r];
      const double wr = s.w[r];
      ay = fma(wr, s.Y[col + i], ay);
      az = fma(wr, s.Z[col + i], az);
    }
  } else if (i < n) {
    for (int r = r0 + w; r < r1; r += 8) {
      const long long col = static_cast<long long>(s.kp) * s.order[r];
      const double wr = s.w[r];
      const double z = (s.mixed == 2) ? static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16*>(s.Zm)[col + i]))
                                      : static_cast<double>(static_cast<const float*>(s.Zm)[col + i]);
      ay = fma(wr, static_cast<double>(s.Y32[col + i]), ay);
      az = fma(wr, z, az);
    }
  }
  shy[w][lane] = ay;
  shz[w][lane] = az;
  __syncthreads();
  if (w == 0 && i < n) {
    double y = 0.0, z = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      y += shy[q][lane];
      z += shz[q][lane];
    }
    s.part[static_cast<long long>(2 * ch) * ldn + i] = y;
    s.part[static_cast<long long>(2 * ch + 1) * ldn + i] = z;
  }
}

__global__ void __launch_bounds__(256) k_recomb_final(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int i = t * 256 + threadIdx.x;
  if (i >= s.n) return;
  const int nch = ceil_div(s.mu, 256);
  double y = 0.0, z = 0.0;
  for (int ch = 0; ch < nch; ++ch) {
    y += s.part[static_cast<long long>(2 * ch) * s.ldn + i];
    z += s.part[static_cast<long long>(2 * ch + 1) * s.ldn + i];
  }
  s.yw[i] = y;
  s.zw[i] = z;
}

void launch_recomb_partial(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_recomb_partial<<<tm.total, 256, 0, st>>>(S, tm);
}
void launch_recomb_final(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_recomb_final<<<tm.total, 256, 0, st>>>(S, tm);
}

// ------------------------ p_sigma: B <z>_w (two stages) ---------------------
__global__ void __launch_bounds__(256) k_psigma_partial(Search* S, TileMap tm) {
  __shared__ double sh[8][33];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn;
  const int nrt = ceil_div(n, 32);
  const int rt = t % nrt, ch = t / nrt;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = rt * 32 + lane;
  const int j1 = min(n, ch * 256 + 256);
  double acc = 0.0;
  if (i < n) {
    for (int j = ch * 256 + w; j < j1; j += 8) acc = fma(s.B[i + static_cast<long long>(ldn) * j], s.zw[j], acc);
  }
  sh[w][lane] = acc;
  __syncthreads();
  if (w == 0 && i < n) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) v += sh[q][lane];
    s.part[static_cast<long long>(ch) * ldn + i] = v;
  }
}

// p_sigma <- (1 - c_s) p_sigma + sqrt(c_s (2 - c_s) mu_eff) B <z>_w
__global__ void __launch_bounds__(256) k_psigma_final(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int i = t * 256 + threadIdx.x;
  if (i >= s.n) return;
  const int nch = ceil_div(s.n, 256);
  double v = 0.0;
  for (int ch = 0; ch < nch; ++ch) v += s.part[static_cast<long long>(ch) * s.ldn + i];
  const double coef = sqrt(s.cs * (2.0 - s.cs) * s.mueff);
  s.ps[i] = (1.0 - s.cs) * s.ps[i] + coef * v;
}

void launch_psigma_partial(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_psigma_partial<<<tm.total, 256, 0, st>>>(S, tm);
}
void launch_psigma_final(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_psigma_final<<<tm.total, 256, 0, st>>>(S, tm);
}

// ------------------------------- finalize -----------------------------------
// ||p_sigma||, h_sigma, p_c, m, sigma, best point, best-f history, generation
// count and whether the eigendecomposition is due. One block per search.
__global__ void __launch_bounds__(256) k_finalize(Search* S, int s0) {
  __shared__ double sh[32];
  Search& s = S[s0 + blockIdx.x];
  if (s.done) return;
  const int n = s.n;
  double sq = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) sq += s.ps[i] * s.ps[i];
  const double psn = sqrt(block_sum<256>(sq, sh));
  const double hs_lhs = psn / sqrt(1.0 - pow(1.0 - s.cs, 2.0 * (s.gen + 1)));
  const double hsig = (hs_lhs < (1.4 + 2.0 / (n + 1.0)) * s.chin) ? 1.0 : 0.0;
  const double pc_coef = hsig * sqrt(s.cc * (2.0 - s.cc) * s.mueff);
  const double sigma = s.sigma;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double y = s.yw[i];
    s.pc[i] = (1.0 - s.cc) * s.pc[i] + pc_coef * y;
    s.m[i] = s.m[i] + sigma * y;
  }
  const int i0 = s.order[0];
  double f0 = s.f[i0];
  double ferr = 0.0;
  if (s.mixed && s.obj != 0) {
    // the value that decides the best point and the history is the FP64 one;
    // its distance from the mixed value that ranked it is kept beside it
    double acc = 0.0;
    for (int t = 0; t < tiles_reeval(n); ++t) acc += s.fpart[t];
    f0 = (s.obj == 2) ? 10.0 * n + acc : acc;
    ferr = fabs(s.f[i0] - f0);
  }
  const bool better = f0 < s.best_f;
  if (better) {
    const double* x = s.X + static_cast<long long>(s.ldn) * i0;
    for (int i = threadIdx.x; i < n; i += 256) s.best_x[i] = x[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.psnorm = psn;
    s.hsig = hsig;
    s.sigma = sigma * exp((s.cs / s.ds) * (psn / s.chin - 1.0));
    if (better) s.best_f = f0;
    s.hist[s.hist_count % s.hist_len] = f0;
    s.hist[s.hist_cap + s.hist_count % s.hist_len] = ferr;
    s.hist_count += 1;
    s.gen += 1;
    s.eig_due = (s.gen % s.g_eig) == 0;
  }
}

void launch_finalize(Search* S, int s0, int s1, DevOptions o, cudaStream_t st) {
  (void)o;
  if (s1 > s0) k_finalize<<<s1 - s0, 256, 0, st>>>(S, s0);
}

// --------------------------- covariance update -------------------------------
// Eq. (2) through Eq. (3): C <- a C + c1 p_c p_c^T + c_mu sum_r w_r y_r y_r^T
// with a = 1 - c1 - c_mu + c1 (1 - h_sigma) c_c (2 - c_c). Only the upper
// 64 x 64 tiles are formed and each writes C(i, j) and its mirror C(j, i), so C
// stays exactly symmetric; reads touch the upper triangle only, which makes the
// in-place update race free. The rank sum is split into chunks of cov_kc
// ranks (k_cov_partial, one CTA per tile and chunk) and the chunk sums are
// added in chunk order by k_cov_reduce, which applies the update. With a
// single chunk the partial kernel applies the update itself.
void cov_split(int n, int mu_cap, int* kc, int* nch) {
  const int tiles = tiles_sym(n);
  const int max_ch = tiles >= 512 ? 1 : 512 / tiles;
  int c = ceil_div(mu_cap, 64);
  if (c > max_ch) c = max_ch;
  if (c < 1) c = 1;
  const int k = ((ceil_div(mu_cap, c) + 15) / 16) * 16;
  *kc = k > 0 ? k : 16;
  *nch = ceil_div(mu_cap, *kc) > 0 ? ceil_div(mu_cap, *kc) : 1;
}

__device__ __forceinline__ void sym_tile(int t, int n, int& ti, int& tj) {
  const int T = ceil_div(n, kGBM);
  int rem = t;
  ti = 0;
  while (rem >= T - ti) { rem -= T - ti; ++ti; }
  tj = ti + rem;
}

__global__ void __launch_bounds__(256) k_cov_partial(Search* S, TileMap tm) {
  __shared__ GemmSmem sm;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn, mu = s.mu, nch = s.cov_nch, kc = s.cov_kc;
  const int tile = t / nch, c = t % nch;
  const int k_lo = c * kc;
  if (k_lo >= mu) return;
  const int k_hi = min(mu, k_lo + kc);
  int ti, tj;
  sym_tile(tile, n, ti, tj);
  const double* Y = s.Y;
  const double* w = s.w + k_lo;
  const int* order = s.order + k_lo;
  if (nch == 1) {
    double* C = s.C;
    const double* pc = s.pc;
    const double c1 = s.c1, cmu = s.cmu;
    const double a = 1.0 - c1 - cmu + c1 * (1.0 - s.hsig) * s.cc * (2.0 - s.cc);
    gemm_tile_f64<true, false>(
        n, n, k_hi - k_lo, ti * kGBM, tj * kGBN,
        [=] __device__(int i, int r) { return w[r] * Y[i + static_cast<long long>(ldn) * order[r]]; },
        [=] __device__(int r, int j) { return Y[j + static_cast<long long>(ldn) * order[r]]; },
        [=] __device__(int i, int j, double acc) {
          if (i > j) return;
          const long long e = i + static_cast<long long>(ldn) * j;
          const double v = a * C[e] + c1 * pc[i] * pc[j] + cmu * acc;
          C[e] = v;
          C[j + static_cast<long long>(ldn) * i] = v;
        },
        sm);
    return;
  }
  double* out = s.covpart + (static_cast<long long>(tile) * nch + c) * (kGBM * kGBN);
  const int i0 = ti * kGBM, j0 = tj * kGBN;
  gemm_tile_f64<true, false>(
      n, n, k_hi - k_lo, i0, j0,
      [=] __device__(int i, int r) { return w[r] * Y[i + static_cast<long long>(ldn) * order[r]]; },
      [=] __device__(int r, int j) { return Y[j + static_cast<long long>(ldn) * order[r]]; },
      [=] __device__(int i, int j, double acc) { out[(i - i0) + kGBM * (j - j0)] = acc; }, sm);
}

__global__ void __launch_bounds__(256) k_cov_reduce(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || s.cov_nch == 1) return;
  const int n = s.n, ldn = s.ldn, nch = s.cov_nch;
  const int used = ceil_div(s.mu, s.cov_kc);
  const int sub = t & 3;  // a quarter of the tile per block
  t >>= 2;
  int ti, tj;
  sym_tile(t, n, ti, tj);
  const double c1 = s.c1, cmu = s.cmu;
  const double a = 1.0 - c1 - cmu + c1 * (1.0 - s.hsig) * s.cc * (2.0 - s.cc);
  const double* part = s.covpart + static_cast<long long>(t) * nch * (kGBM * kGBN);
  for (int e = sub * 1024 + threadIdx.x; e < (sub + 1) * 1024; e += 256) {
    const int ii = e & (kGBM - 1), jj = e >> 6;
    const int i = ti * kGBM + ii, j = tj * kGBN + jj;
    if (i >= n || j >= n || i > j) continue;
    double acc = 0.0;
    for (int c = 0; c < used; ++c) acc += part[static_cast<long long>(c) * (kGBM * kGBN) + e];
    const long long x = i + static_cast<long long>(ldn) * j;
    const double v = a * s.C[x] + c1 * s.pc[i] * s.pc[j] + cmu * acc;
    s.C[x] = v;
    s.C[j + static_cast<long long>(ldn) * i] = v;
  }
}

void launch_cov_partial(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_cov_partial<<<tm.total, 256, 0, st>>>(S, tm);
}
void launch_cov_reduce(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_cov_reduce<<<tm.total, 256, 0, st>>>(S, tm);
}

// ------------------------------ stop + restart ------------------------------
// Stop tests of §2.2 (constants after Auger & Hansen 2005), then Algorithm 2:
// the search ends when the target is reached or the restart budget is spent,
// otherwise a new descent starts with lambda doubled (or kept), a uniform
// mean in the box, and C = B = I. The products and sums that decide a flag are
// rounded separately (no contraction) to match a plain evaluation.
template <int NT>
__device__ void restart_descent(Search& s, const DevOptions& o, double* sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    s.restart += 1;
    if (o.ipop_double) s.lam *= 2;
  }
  __syncthreads();
  reset_descent<NT>(s);
  for (int i = threadIdx.x; i < s.n; i += NT)
    s.m[i] = restart_mean_coord(i, s.index, s.restart, o.key0, o.key1, o.box_lo, o.box_hi);
  __syncthreads();
  compute_params<NT>(s, o, sh);
}

__global__ void __launch_bounds__(256) k_stop(Search* S, int s0, DevOptions o) {
  __shared__ double sh[32];
  __shared__ int shi[32];
  Search& s = S[s0 + blockIdx.x];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn;
  const double sigma = s.sigma;
  const double tolx = o.tol_x_factor * s.sigma0;
  const int j = s.gen % n;
  const double axis = __dmul_rn(__dmul_rn(0.1, sigma), s.D[j]);
  const double coord = __dmul_rn(0.2, sigma);
  int tolx_fail = 0, axis_moves = 0, coord_stuck = 0, nonfinite = 0;
  double dmax = 0.0, dmin = INFINITY;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double cii = s.C[i + static_cast<long long>(ldn) * i];
    const double sd = sqrt(fmax(cii, 0.0));
    const double mi = s.m[i];
    if (!(__dmul_rn(sigma, fabs(s.pc[i])) < tolx) || !(__dmul_rn(sigma, sd) < tolx)) tolx_fail = 1;
    if (__dadd_rn(mi, __dmul_rn(axis, s.B[i + static_cast<long long>(ldn) * j])) != mi) axis_moves = 1;
    if (__dadd_rn(mi, __dmul_rn(coord, sd)) == mi) coord_stuck = 1;
    if (!isfinite(mi) || !isfinite(cii)) nonfinite = 1;
    dmax = fmax(dmax, s.D[i]);
    dmin = fmin(dmin, s.D[i]);
  }
  const int any_tolx_fail = block_or<256>(tolx_fail, shi);
  const int any_axis_moves = block_or<256>(axis_moves, shi);
  const int any_coord_stuck = block_or<256>(coord_stuck, shi);
  const int any_nonfinite = block_or<256>(nonfinite, shi);
  dmax = block_max<256>(dmax, sh);
  dmin = -block_max<256>(-dmin, sh);
  int flags = 0;
  if (threadIdx.x == 0) {
    if (s.best_f < o.f_target) flags |= 1;
    if (s.gen >= s.max_iter) flags |= 2;
    if (s.hist_count >= s.hist_len) {
      // TolHistFun; on a mixed handle the range is compared with at least
      // kMixedResolution times the largest mixed-evaluation error of the
      // window's best values (below that the mixed ranking cannot tell the
      // candidates apart, so the descent cannot make further progress)
      double hmax = -INFINITY, hmin = INFINITY, emax = 0.0;
      for (int q = 0; q < s.hist_len; ++q) {
        hmax = fmax(hmax, s.hist[q]);
        hmin = fmin(hmin, s.hist[q]);
        emax = fmax(emax, s.hist[s.hist_cap + q]);
      }
      if (hmax - hmin < fmax(o.tol_hist_fun, kMixedResolution * emax)) flags |= 4;
    }
    if (!any_tolx_fail) flags |= 8;
    if (__dmul_rn(dmax, dmax) > __dmul_rn(__dmul_rn(o.cond_max, dmin), dmin)) flags |= 16;
    if (!any_axis_moves) flags |= 32;
    if (any_coord_stuck) flags |= 64;
    if (any_nonfinite || !isfinite(sigma)) {
      flags |= 128;
      atomicOr(s.err, kDevErrNonFinite);  // reported to the host as CMAES_ENUMERIC
    }
    flags &= o.stop_mask;
    s.flags = flags;
    shi[0] = flags;
  }
  __syncthreads();
  flags = shi[0];
  __syncthreads();
  if (!flags) return;
  // a restart that would outgrow the panels allocated for lambda ends the search
  if ((flags & 1) || s.restart + 1 > o.max_restarts || (o.ipop_double && 2 * s.lam > s.lam_cap)) {
    if (threadIdx.x == 0) s.done = 1;
    return;
  }
  if (o.restart_hold) {  // the host decides when (and whether) this search restarts
    if (threadIdx.x == 0) s.done = 2;
    return;
  }
  restart_descent<256>(s, o, sh);
}

void launch_stop(Search* S, int s0, int s1, DevOptions o, cudaStream_t st) {
  if (s1 > s0) k_stop<<<s1 - s0, 256, 0, st>>>(S, s0, o);
}

__global__ void __launch_bounds__(256) k_force_restart(Search* S, int si, DevOptions o) {
  __shared__ double sh[32];
  if (threadIdx.x == 0) S[si].done = 0;  // resumes a paused search (restart_hold)
  restart_descent<256>(S[si], o, sh);
}

void launch_force_restart(Search* S, int s, DevOptions o, cudaStream_t st) {
  k_force_restart<<<1, 256, 0, st>>>(S, s, o);
}

}  // namespace cmaes_gb300
