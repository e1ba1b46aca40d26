// kernels_mixed.cu -- the mixed-precision GEMMs of a generation on the
// tcgen05 tensor cores (TF32 or BF16 inputs, FP32 accumulation in TMEM).
//
//   k_tc_sample     Eq. (1) as one GEMM (§3.1): Y = (B D) Z with the operands in
//                   TF32/BF16, then x = m + sigma y formed in FP64.
//   k_tc_objective  U^T = (X - x*)^T Q^T with 3-term split operands
//                   (hi*hi + hi*lo + lo*hi, about 22 significant bits), x - x*
//                   formed in FP64; each thread owns one candidate and sums
//                   its objective terms straight from TMEM in FP32 (Kahan
//                   summation): Lambda_i u_i^2 for the ellipsoid, and for the
//                   Rastrigin u_i^2 + 20 sin^2(pi u_i), which equals
//                   u_i^2 - 10 cos(2 pi u_i) + 10 and keeps its relative
//                   accuracy near the optimum (GB300's FP64 pipe is 1/64 of
//                   the FP32 one, so FP64 transcendentals here would dominate).
//   k_tc_cov_*      the rank-mu sum of Eq. (3), sum_r w_r y_r y_r^T, with split
//                   operands (the FP32-accuracy correction term), upper
//                   128 x 128 tiles, rank chunks added in order in FP64.
//   k_reeval        the FP64 value of each generation's best point, so the
//                   target test and the best-so-far record never rest on a
//                   mixed-precision value.
// The eigendecomposition, the mean, the paths and sigma stay FP64.
#include <cmath>
#include "device_common.cuh"
#include "tc_common.cuh"

namespace cmaes_gb300 {

int tc_elem_bytes(int precision) { return precision == 2 ? 2 : 4; }
int tiles_tc_sample(int n, int lam_cap) { return ceil_div(n, 128) * ceil_div(lam_cap, 256); }
int tiles_tc_objective(int lam_cap) { return ceil_div(lam_cap, 128); }
int tiles_tc_sym(int n) {
  const int t = ceil_div(n, 128);
  return t * (t + 1) / 2;
}
void tc_cov_split(int n, int mu_cap, int* kc, int* nch) {
  const int tiles = tiles_tc_sym(n);
  const int max_ch = tiles >= 304 ? 1 : 304 / tiles;
  int c = ceil_div(mu_cap, 128);
  if (c > max_ch) c = max_ch;
  if (c < 1) c = 1;
  const int k = ((ceil_div(mu_cap, c) + 31) / 32) * 32;
  *kc = k > 0 ? k : 32;
  *nch = ceil_div(mu_cap, *kc) > 0 ? ceil_div(mu_cap, *kc) : 1;
}

namespace {

template <int KIND>
using ET = typename TcElem<KIND>::T;

__device__ __forceinline__ void sym_tile128(int t, int n, int& ti, int& tj) {
  const int T = ceil_div(n, 128);
  int rem = t;
  ti = 0;
  while (rem >= T - ti) { rem -= T - ti; ++ti; }
  tj = ti + rem;
}

// 16-byte vector of epv input-format values
template <int KIND>
struct __align__(16) Vec16 {
  static constexpr int epv = 16 / TcElem<KIND>::esz;
  ET<KIND> v[epv];
};

}  // namespace

// ------------------------------ preparation ---------------------------------
// Q rows in the input format (hi and lo parts), K-major, zero beyond n.
template <int KIND>
__global__ void __launch_bounds__(256) k_tc_prepare_q(Search* S, int si) {
  const Search& s = S[si];
  const int n = s.n, kp = s.kp, ldn = s.ldn;
  ET<KIND>* qh = static_cast<ET<KIND>*>(s.QTh);
  ET<KIND>* ql = static_cast<ET<KIND>*>(s.QTl);
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < static_cast<long long>(n) * kp; e += 256LL * gridDim.x) {
    const int i = static_cast<int>(e / kp), k = static_cast<int>(e % kp);
    ET<KIND> h = TcElem<KIND>::from(0.0f), l = TcElem<KIND>::from(0.0f);
    if (k < n) tc_split<KIND>(s.Q[i + static_cast<long long>(ldn) * k], h, l);
    qh[e] = h;
    ql[e] = l;
    if (k == 0) s.lam32[i] = static_cast<float>(s.lamdiag[i]);
  }
}

void launch_tc_prepare_q(Search* S, int s, int precision, cudaStream_t st) {
  if (precision == 2) k_tc_prepare_q<1><<<152, 256, 0, st>>>(S, s);
  else k_tc_prepare_q<0><<<152, 256, 0, st>>>(S, s);
}

// BDT(i, k) = B(i, k) D(k) in the input format, through a shared-memory
// transpose of 64 x 64 tiles (coalesced on both sides); with with_bd the same
// values also go to BD in FP64 (the eigendecomposition's B diag(D)).
template <int KIND>
__global__ void __launch_bounds__(256) k_tc_set_bdt(Search* S, TileMap tm, int force, int with_bd) {
  __shared__ double tile[64][65];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !(force || s.eig_due)) return;
  const int n = s.n, ldn = s.ldn, kp = s.kp, T = ceil_div(n, 64);
  const int i0 = (t % T) * 64, k0 = (t / T) * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int ii = e & 63, kk = e >> 6;
    const int i = i0 + ii, k = k0 + kk;
    const bool in = i < n && k < n;
    const double v = in ? s.B[i + static_cast<long long>(ldn) * k] * s.D[k] : 0.0;
    tile[kk][ii] = v;
    if (with_bd && in) s.BD[i + static_cast<long long>(ldn) * k] = v;  // BD = B diag(D) in FP64
  }
  __syncthreads();
  ET<KIND>* bdt = static_cast<ET<KIND>*>(s.BDT);
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int kk = e & 63, ii = e >> 6;
    const int i = i0 + ii, k = k0 + kk;
    if (i < n && k < n) bdt[static_cast<long long>(i) * kp + k] = TcElem<KIND>::from(static_cast<float>(tile[kk][ii]));
  }
}

void launch_tc_set_bdt(Search* S, TileMap tm, int precision, int force, cudaStream_t st) {
  if (tm.total <= 0) return;
  if (precision == 2) k_tc_set_bdt<1><<<tm.total, 256, 0, st>>>(S, tm, force, 0);
  else k_tc_set_bdt<0><<<tm.total, 256, 0, st>>>(S, tm, force, 0);
}

void launch_tc_set_bd_bdt(Search* S, TileMap tm, int precision, cudaStream_t st) {
  if (tm.total <= 0) return;
  if (precision == 2) k_tc_set_bdt<1><<<tm.total, 256, 0, st>>>(S, tm, 0, 1);
  else k_tc_set_bdt<0><<<tm.total, 256, 0, st>>>(S, tm, 0, 1);
}

// -------------------------------- sampling ----------------------------------
// Tile: 128 rows of Y by 256 candidates, K = kp (zero padded).
template <int KIND>
__global__ void __launch_bounds__(256, 1) k_tc_sample(Search* S, TileMap tm) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, kp = s.kp, lam = s.lam, ldn = s.ldn, lam_cap = s.lam_cap;
  const int mt = ceil_div(n, 128);
  const int i0 = (t % mt) * 128, j0 = (t / mt) * 256;
  if (j0 >= lam) return;
  TcCtx ctx;
  tc_begin(ctx, dyn, mbar, &tslot);
  constexpr int epv = Vec16<KIND>::epv, esz = TcElem<KIND>::esz, vpr = kTcKC / epv;
  const char* bdt = static_cast<const char*>(s.BDT);
  const char* zm = static_cast<const char*>(s.Zm);
  auto stage = [&](int k0, unsigned char* a_hi, unsigned char*, unsigned char* b_hi, unsigned char*) {
    for (int e = threadIdx.x; e < 128 * vpr; e += 256) {
      const int r = e / vpr, v = e % vpr, i = i0 + r, k = k0 + v * epv;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (i < n) val = *reinterpret_cast<const uint4*>(bdt + (static_cast<long long>(i) * kp + k) * esz);
      *reinterpret_cast<uint4*>(a_hi + tc_off<KIND>(r, v * epv)) = val;
    }
    for (int e = threadIdx.x; e < 256 * vpr; e += 256) {
      const int r = e / vpr, v = e % vpr, j = j0 + r, k = k0 + v * epv;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (j < lam_cap) val = *reinterpret_cast<const uint4*>(zm + (static_cast<long long>(j) * kp + k) * esz);
      *reinterpret_cast<uint4*>(b_hi + tc_off<KIND>(r, v * epv)) = val;
    }
  };
  const bool ok = tc_tile<KIND, false>(ctx, 256, kp, stage);
  if (ok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int i = i0 + quarter * 32 + lane;
    const double mi = (i < n) ? s.m[i] : 0.0;
    const double sigma = s.sigma;
    for (int c = half * 128; c < half * 128 + 128; c += 16) {
      float v[16];
      tmem_ld16(ctx.tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = j0 + c + q;
        if (i < n && j < lam) {
          s.Y32[static_cast<long long>(j) * kp + i] = v[q];
          s.X[i + static_cast<long long>(ldn) * j] = mi + sigma * static_cast<double>(v[q]);
        }
      }
    }
  }
  tc_end(ctx);
  if (!ok && threadIdx.x == 0) atomicOr(s.err, 1);
}

void tc_set_attributes_once();

void launch_tc_sample(Search* S, TileMap tm, int precision, cudaStream_t st) {
  if (tm.total <= 0) return;
  tc_set_attributes_once();
  if (precision == 2)
    k_tc_sample<1><<<tm.total, 256, TcPlan<1, false>::bytes, st>>>(S, tm);
  else
    k_tc_sample<0><<<tm.total, 256, TcPlan<0, false>::bytes, st>>>(S, tm);
}

// -------------------------------- objective ---------------------------------
// Tile: 128 candidates; loops over 256-row blocks of Q. D(j, i) = u_i of
// candidate j; thread (quarter, lane) owns candidate j, its warp half owns
// half of the tile's columns.
template <int KIND>
__global__ void __launch_bounds__(256, 1) k_tc_objective(Search* S, TileMap tm) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ double fsum[2][128];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || s.obj == 3) return;
  const int n = s.n, kp = s.kp, lam = s.lam, ldn = s.ldn, lam_cap = s.lam_cap;
  const int j0 = t * 128;
  if (j0 >= lam) return;
  TcCtx ctx;
  tc_begin(ctx, dyn, mbar, &tslot);
  constexpr int epv = Vec16<KIND>::epv, esz = TcElem<KIND>::esz, vpr = kTcKC / epv;
  const char* qh = static_cast<const char*>(s.QTh);
  const char* ql = static_cast<const char*>(s.QTl);
  const double* X = s.X;
  const double* xs = s.xstar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  float facc = 0.0f, fcomp = 0.0f;  // Kahan sum
  const float* lam32 = s.lam32;
  const bool ellipsoid = s.obj == 1;
  bool ok = true;
  for (int r0 = 0; r0 < n && ok; r0 += 256) {
    const int nt = min(256, ((n - r0 + 15) / 16) * 16);
    auto stage = [&](int k0, unsigned char* a_hi, unsigned char* a_lo, unsigned char* b_hi, unsigned char* b_lo) {
      for (int e = threadIdx.x; e < 128 * vpr; e += 256) {
        const int r = e / vpr, v = e % vpr, j = j0 + r, k = k0 + v * epv;
        Vec16<KIND> h, l;
#pragma unroll
        for (int q = 0; q < epv; ++q) {
          float d = 0.0f;  // x - x* formed in FP64, split in FP32
          if (j < lam_cap && k + q < n) d = static_cast<float>(X[(k + q) + static_cast<long long>(ldn) * j] - xs[k + q]);
          tc_split32<KIND>(d, h.v[q], l.v[q]);
        }
        *reinterpret_cast<Vec16<KIND>*>(a_hi + tc_off<KIND>(r, v * epv)) = h;
        *reinterpret_cast<Vec16<KIND>*>(a_lo + tc_off<KIND>(r, v * epv)) = l;
      }
      for (int e = threadIdx.x; e < nt * vpr; e += 256) {
        const int r = e / vpr, v = e % vpr, i = r0 + r, k = k0 + v * epv;
        uint4 vh = make_uint4(0, 0, 0, 0), vl = make_uint4(0, 0, 0, 0);
        if (i < n) {
          const long long off = (static_cast<long long>(i) * kp + k) * esz;
          vh = *reinterpret_cast<const uint4*>(qh + off);
          vl = *reinterpret_cast<const uint4*>(ql + off);
        }
        *reinterpret_cast<uint4*>(b_hi + tc_off<KIND>(r, v * epv)) = vh;
        *reinterpret_cast<uint4*>(b_lo + tc_off<KIND>(r, v * epv)) = vl;
      }
    };
    ok = tc_tile<KIND, true>(ctx, nt, kp, stage);
    if (!ok) break;
    const int c_hi = min(half * 128 + 128, nt);
    for (int c = half * 128; c < c_hi; c += 16) {
      float v[16];
      tmem_ld16(ctx.tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = r0 + c + q;
        if (i < n) {
          const float u = v[q];
          float term;
          if (ellipsoid) {
            term = lam32[i] * u * u;
          } else {
            const float sp = sinpif(u);
            term = u * u + 20.0f * sp * sp;
          }
          const float y = term - fcomp;
          const float t2 = facc + y;
          fcomp = (t2 - facc) - y;
          facc = t2;
        }
      }
    }
    tc_tile_done();
  }
  fsum[half][quarter * 32 + lane] = static_cast<double>(facc) - static_cast<double>(fcomp);
  __syncthreads();
  if (ok && half == 0) {
    const int j = j0 + quarter * 32 + lane;
    if (j < lam) s.f[j] = fsum[0][quarter * 32 + lane] + fsum[1][quarter * 32 + lane];
  }
  tc_end(ctx);
  if (!ok && threadIdx.x == 0) atomicOr(s.err, 1);
}

void launch_tc_objective(Search* S, TileMap tm, int precision, cudaStream_t st) {
  if (tm.total <= 0) return;
  tc_set_attributes_once();
  if (precision == 2)
    k_tc_objective<1><<<tm.total, 256, TcPlan<1, true>::bytes, st>>>(S, tm);
  else
    k_tc_objective<0><<<tm.total, 256, TcPlan<0, true>::bytes, st>>>(S, tm);
}

// ---------------------------- rank-mu update --------------------------------
// Partial tile (ti, tj) of sum_r w_r y_r y_r^T over ranks [k_lo, k_hi).
template <int KIND>
__global__ void __launch_bounds__(256, 1) k_tc_cov_partial(Search* S, TileMap tm) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, kp = s.kp, mu = s.mu, nch = s.covm_nch, kc = s.covm_kc;
  const int tile = t / nch, c = t % nch;
  const int k_lo = c * kc;
  if (k_lo >= mu) return;
  const int k_hi = min(mu, k_lo + kc);
  int ti, tj;
  sym_tile128(tile, n, ti, tj);
  TcCtx ctx;
  tc_begin(ctx, dyn, mbar, &tslot);
  constexpr int epv = Vec16<KIND>::epv;
  const float* Y = s.Y32;
  const float* w = s.w32;
  const int* order = s.order;
  auto stage = [&](int k0, unsigned char* a_hi, unsigned char* a_lo, unsigned char* b_hi, unsigned char* b_lo) {
    // element (row, rank): rows run over lanes so that each load of a
    // selected column is coalesced
    for (int e = threadIdx.x; e < 128 * (kTcKC / epv); e += 256) {
      const int r = e & 127, v = e >> 7;
      const int ia = ti * 128 + r, ib = tj * 128 + r;
      Vec16<KIND> ah, al, bh, bl;
#pragma unroll
      for (int q = 0; q < epv; ++q) {
        const int rk = k_lo + k0 + v * epv + q;
        float ya = 0.0f, yb = 0.0f;
        if (rk < k_hi) {
          const long long col = static_cast<long long>(order[rk]) * kp;
          if (ia < n) ya = w[rk] * Y[col + ia];
          if (ib < n) yb = Y[col + ib];
        }
        tc_split32<KIND>(ya, ah.v[q], al.v[q]);
        tc_split32<KIND>(yb, bh.v[q], bl.v[q]);
      }
      *reinterpret_cast<Vec16<KIND>*>(a_hi + tc_off<KIND>(r, v * epv)) = ah;
      *reinterpret_cast<Vec16<KIND>*>(a_lo + tc_off<KIND>(r, v * epv)) = al;
      *reinterpret_cast<Vec16<KIND>*>(b_hi + tc_off<KIND>(r, v * epv)) = bh;
      *reinterpret_cast<Vec16<KIND>*>(b_lo + tc_off<KIND>(r, v * epv)) = bl;
    }
  };
  const bool ok = tc_tile<KIND, true>(ctx, 128, k_hi - k_lo, stage);
  if (ok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;
    double* out = s.covpart + (static_cast<long long>(tile) * nch + c) * (128 * 128);
    for (int cc = half * 64; cc < half * 64 + 64; cc += 16) {
      float v[16];
      tmem_ld16(ctx.tmem + (static_cast<uint32_t>(quarter * 32) << 16) + cc, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) out[r + 128 * (cc + q)] = static_cast<double>(v[q]);
    }
  }
  tc_end(ctx);
  if (!ok && threadIdx.x == 0) atomicOr(s.err, 1);
}

void launch_tc_cov_partial(Search* S, TileMap tm, int precision, cudaStream_t st) {
  if (tm.total <= 0) return;
  tc_set_attributes_once();
  if (precision == 2)
    k_tc_cov_partial<1><<<tm.total, 256, TcPlan<1, true>::bytes, st>>>(S, tm);
  else
    k_tc_cov_partial<0><<<tm.total, 256, TcPlan<0, true>::bytes, st>>>(S, tm);
}

// The dynamic shared memory of the six tensor-core GEMM kernels, set at the
// first launch of any of them (the per-generation graphs replay the launches
// without coming back here).
void tc_set_attributes_once() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_tc_sample<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<0, false>::bytes);
  cudaFuncSetAttribute(k_tc_sample<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<1, false>::bytes);
  cudaFuncSetAttribute(k_tc_objective<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<0, true>::bytes);
  cudaFuncSetAttribute(k_tc_objective<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<1, true>::bytes);
  cudaFuncSetAttribute(k_tc_cov_partial<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<0, true>::bytes);
  cudaFuncSetAttribute(k_tc_cov_partial<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcPlan<1, true>::bytes);
  done = true;
}

// C <- a C + c1 p_c p_c^T + c_mu (sum of the chunk partials, in chunk order),
// upper 128 x 128 tiles with mirror writes.
__global__ void __launch_bounds__(256) k_tc_cov_reduce(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done) return;
  const int n = s.n, ldn = s.ldn, nch = s.covm_nch;
  const int used = ceil_div(s.mu, s.covm_kc);
  const int sub = t & 15;  // a sixteenth of the tile per block
  t >>= 4;
  int ti, tj;
  sym_tile128(t, n, ti, tj);
  const double c1 = s.c1, cmu = s.cmu;
  const double a = 1.0 - c1 - cmu + c1 * (1.0 - s.hsig) * s.cc * (2.0 - s.cc);
  const double* part = s.covpart + static_cast<long long>(t) * nch * (128 * 128);
  for (int e = sub * 1024 + threadIdx.x; e < (sub + 1) * 1024; e += 256) {
    const int r = e & 127, cc = e >> 7;
    const int i = ti * 128 + r, j = tj * 128 + cc;
    if (i >= n || j >= n || i > j) continue;
    double acc = 0.0;
    for (int c = 0; c < used; ++c) acc += part[static_cast<long long>(c) * (128 * 128) + e];
    const long long x = i + static_cast<long long>(ldn) * j;
    const double v = a * s.C[x] + c1 * s.pc[i] * s.pc[j] + cmu * acc;
    s.C[x] = v;
    s.C[j + static_cast<long long>(ldn) * i] = v;
  }
}

void launch_tc_cov_reduce(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_tc_cov_reduce<<<tm.total, 256, 0, st>>>(S, tm);
}

// ---------------------- FP64 value of the best point ------------------------
// Rows [32 t, 32 t + 32) of u = Q (x - x*) for x = X[:, order[0]]: lane = row
// (coalesced along Q's columns), the eight warps take eight segments of k, and
// warp 0 adds the segments in order, forms the objective terms of its rows and
// sums them in a fixed order into fpart[t].
__global__ void __launch_bounds__(256) k_reeval(Search* S, TileMap tm) {
  __shared__ double part[8][33];
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !s.mixed || s.obj == 0) return;
  const int n = s.n, ldn = s.ldn;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = t * 32 + lane;
  const double* x = s.X + static_cast<long long>(ldn) * s.order[0];
  const int kseg = ceil_div(n, 8), k0 = warp * kseg, k1 = min(n, k0 + kseg);
  double u = 0.0;
  if (i < n && s.obj != 3)
    for (int k = k0; k < k1; ++k) u = fma(s.Q[i + static_cast<long long>(ldn) * k], x[k] - s.xstar[k], u);
  part[warp][lane] = u;
  __syncthreads();
  if (warp != 0) return;
  double g = 0.0;
  if (i < n) {
    if (s.obj == 3) {
      const double r = x[i] - s.xstar[i];
      g = r * r;
    } else {
      double uu = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) uu += part[w][lane];
      g = (s.obj == 1) ? s.lamdiag[i] * uu * uu : uu * uu - 10.0 * cos((2.0 * 3.141592653589793) * uu);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
  if (lane == 0) s.fpart[t] = g;
}

void launch_reeval(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_reeval<<<tm.total, 256, 0, st>>>(S, tm);
}

}  // namespace cmaes_gb300
