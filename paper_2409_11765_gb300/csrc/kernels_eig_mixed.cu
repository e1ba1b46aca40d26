// kernels_eig_mixed.cu -- mixed-precision route of the warm-started
// eigendecomposition (32 < n <= kEigBigMaxN, every handle precision: the FP32
// work only supplies the starting basis, the result is FP64-accurate). The
// FP32 Jacobi here runs in one CTA (n <= kEigMixedMaxN); above that size it is
// the many-CTA form of kernels_eig_big.cu, and the rest is shared.
//
// The FP64 Jacobi of kernels_eig.cu / kernels_jacobi_cluster.cu needs about
// seven sweeps per decomposition when C moves a lot between generations, and on
// GB300 every sweep is bound by the FP64 pipe (1/64 of the FP32 rate) and by
// the latency of its steps. Here the sweeps run in FP32 and FP64 accuracy is
// recovered by dense FP64 products that spread over every SM:
//   1. A = B^T C B in FP64 (the warm start, from the previous basis B), and
//      A32 = A - c I in FP32 with c = trace(A) / n.
//   2. FP32 cyclic Jacobi on A32 (round-robin ordering, the rotation of
//      Golub & Van Loan §8.5) down to FP32 resolution in one CTA per search;
//      it logs its rotations, and V32 = their product is formed from the log
//      by one warp per row across the GPU. X0 = B V32 in FP64 is an
//      orthonormal basis to ~1e-7 whose columns are eigenvectors of C to FP32
//      accuracy.
//   3. Two steps of the iterative refinement of Ogita & Aishima ("Iterative
//      refinement for symmetric eigenvalue decomposition", Japan J. Indust.
//      Appl. Math. 35, 2018): with S = X^T C X, G = X^T X, lambda_i = s_ii / g_ii,
//        e_ii = (1 - g_ii) / 2,
//        e_ij = (s_ij - lambda_j g_ij) / (lambda_j - lambda_i)   (i != j),
//        X <- X + X E,
//      the first-order correction that makes X orthonormal and C-diagonal
//      together; the error squares at every step. A pair whose correction
//      would exceed 2^-10 (eigenvalues too close for first order) only gets the
//      orthogonality part e_ij = -g_ij / 2 and is left to step 5.
//   4. One Newton-Schulz step X <- X + X (I - X^T X) / 2 removes the
//      second-order loss of orthogonality that large first-order corrections
//      leave (error e -> 1.5 e^2).
//   5. A = X^T C X in FP64, B <- X; on mixed-precision handles a few rounds of
//      targeted rotations (k_pair_rounds) take the pairs the refinement left;
//      the FP64 Jacobi then runs on (A, B) as in
//      the FP64 path: it rotates what step 3 left (pairs of close eigenvalues),
//      normally ends at its first quiet step, and delivers the eigenvalues, the
//      PD guard and the canonical form. Off-diagonal entries below
//      n eps64 max|a_ii| (FP64 handles) or 4 n eps64 max|a_ii| (mixed
//      handles), the rounding level of the product that formed A, are left
//      alone.
// Because X^T X is measured and corrected every decomposition, rounding does
// not accumulate in B from one generation's warm start to the next.
// Every FP64 product reads its left operand along its leading dimension
// (each X is also stored transposed) and computes 256 consecutive outputs of
// the n x n result per CTA, two per lane, over the full K.
#include <cmath>
#include "device_common.cuh"

namespace cmaes_gb300 {

constexpr int kE32Max = kEigMixedMaxN;  // FP32 Jacobi keeps A32 in shared memory
constexpr int kJ32NT = 1024;
constexpr float kJ32Tol = 1e-6f;

__device__ __forceinline__ bool mixed_route_due(const Search& s) {
  return !s.done && s.eig_due && eig_refined_route(s);
}
// the one-CTA FP32 Jacobi, its log replay and the shared-memory pair rounds
__device__ __forceinline__ bool small_route_due(const Search& s) { return mixed_route_due(s) && s.n <= kE32Max; }

// ---------------------------------------------------------------------------
// FP64 products of the refinement: CTA t of a search computes outputs
// o = t * 256 + warp * 64 + lane + 32 u (u = 0, 1) of the n x n result in
// column-major order, each over the full K = n. The left operand is read along
// its leading dimension (consecutive lanes, consecutive rows), the right one is
// shared by the lanes of a column. FP64 issues at 1/64 of the FP32 rate, so
// batches of loaded operands and independent accumulators keep the pipe busy
// without staging the operands in shared memory; they stay in L1 / L2 up to
// n ~ 1000 (above it the products stream from L2 and HBM).
// ---------------------------------------------------------------------------
constexpr int kFW = 4;               // warps per CTA
constexpr int kFP = 2;               // outputs per lane
constexpr int kFO = kFW * 32 * kFP;  // outputs per CTA
constexpr int kFK = 4;               // k values per batch of the load pipeline
constexpr int kFOS = kFW * 32;       // outputs per CTA of a symmetric product (one per lane)
int tiles_flat(int n) { return ceil_div(n * n, kFO); }
int tiles_flat_sym(int n) { return ceil_div(n * (n + 1) / 2, kFOS); }

// Column j of the packed upper triangle holds outputs o in [j (j+1)/2, (j+1) (j+2)/2).
__device__ __forceinline__ void upper_index(int o, int& i, int& j) {
  int c = static_cast<int>((sqrtf(static_cast<float>(8 * o + 1)) - 1.0f) * 0.5f);
  while ((c + 1) * (c + 2) / 2 <= o) ++c;
  while (c * (c + 1) / 2 > o) --c;
  j = c;
  i = o - c * (c + 1) / 2;
}

// SYM: the result is symmetric (X^T C X, X^T X); only i <= j is computed (in
// packed column order, one output per lane so that the halved work still fills
// as many CTAs) and the epilogue is called for (i, j) and (j, i).
template <int NACC, bool SYM = false, class LA, class LB, class EPI>
__device__ __forceinline__ void gemm_flat_f64(int n, int t, const LA& la, const LB& lb, const EPI& epi) {
  constexpr int kFP = SYM ? 1 : cmaes_gb300::kFP;
  constexpr int kFO = kFW * 32 * kFP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = t * kFO + warp * 32 * kFP + lane;
  const int nn = SYM ? n * (n + 1) / 2 : n * n;
  int ii[kFP], jj[kFP];
#pragma unroll
  for (int u = 0; u < kFP; ++u) {
    const int o = base + 32 * u;
    if (o >= nn) {  // lanes past the end compute (0, 0) and store nothing
      ii[u] = 0;
      jj[u] = 0;
    } else if (SYM) {
      upper_index(o, ii[u], jj[u]);
    } else {
      ii[u] = o % n;
      jj[u] = o / n;
    }
  }
  double acc[NACC][kFP];
#pragma unroll
  for (int a = 0; a < NACC; ++a)
#pragma unroll
    for (int u = 0; u < kFP; ++u) acc[a][u] = 0.0;
  // software pipeline over batches of kFK consecutive k: the operands of the
  // next batch are loaded before the FMAs of the current one, so L2 latency
  // overlaps FP64 work
  double xa0[kFK][kFP], xb0[kFK][NACC][kFP], xa1[kFK][kFP], xb1[kFK][NACC][kFP];
  auto load = [&](double (&xa)[kFK][kFP], double (&xb)[kFK][NACC][kFP], int k0) {
#pragma unroll
    for (int kk = 0; kk < kFK; ++kk)
#pragma unroll
      for (int u = 0; u < kFP; ++u) {
        xa[kk][u] = la(ii[u], k0 + kk);
#pragma unroll
        for (int a = 0; a < NACC; ++a) xb[kk][a][u] = lb(a, k0 + kk, jj[u]);
      }
  };
  auto fmas = [&](const double (&xa)[kFK][kFP], const double (&xb)[kFK][NACC][kFP]) {
#pragma unroll
    for (int kk = 0; kk < kFK; ++kk)
#pragma unroll
      for (int u = 0; u < kFP; ++u)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a][u] = fma(xa[kk][u], xb[kk][a][u], acc[a][u]);
  };
  const int nb = n / kFK;  // full batches; the two register buffers alternate
  if (nb > 0) load(xa0, xb0, 0);
  int b = 0;
  for (; b + 1 < nb; b += 2) {
    load(xa1, xb1, (b + 1) * kFK);
    fmas(xa0, xb0);
    if (b + 2 < nb) load(xa0, xb0, (b + 2) * kFK);
    fmas(xa1, xb1);
  }
  if (b < nb) fmas(xa0, xb0);
  for (int k = nb * kFK; k < n; ++k)
#pragma unroll
    for (int u = 0; u < kFP; ++u) {
      const double x = la(ii[u], k);
#pragma unroll
      for (int a = 0; a < NACC; ++a) acc[a][u] = fma(x, lb(a, k, jj[u]), acc[a][u]);
    }
#pragma unroll
  for (int u = 0; u < kFP; ++u)
    if (base + 32 * u < nn) {
      epi(ii[u], jj[u], acc[0][u], acc[NACC - 1][u]);
      if (SYM && ii[u] != jj[u]) epi(jj[u], ii[u], acc[0][u], acc[NACC - 1][u]);
    }
}

// Buffers of the refinement (ldn x n, FP64): EA, ET, EX, EG, EH plus B.
enum OaOp {
  OA_W0 = 0,  // (C B)^T                    -> EG   (warm start, C symmetric)
  OA_W1,      // A = (C B)^T B = B^T C B    -> EH
  OA_X0,      // X0 = B V32 (V32 in EG)     -> ET, X0^T -> EX
  OA_T0,      // T0 = C X0 (ET)             -> EA
  OA_SG0,     // S0 = X0^T T0, G0 = X0^T X0 -> EG, EH   (X0^T in EX)
  OA_E0,      // E0 from (EG, EH)           -> EA
  OA_U0,      // X1 = X0 + X0 E0            -> EG, X1^T -> EH
  OA_T1,      // T1 = C X1 (EG)             -> EA
  OA_SG1,     // S1, G1 (X1^T in EH)        -> ET, EX
  OA_E1,      // E1 from (ET, EX)           -> EA
  OA_U1,      // X2 = X1 + X1 E1            -> B, X2^T -> ET
  OA_G2,      // M = (I - X2^T X2) / 2      -> EX
  OA_N2,      // X3 = X2 + X2 M             -> EG, X3^T -> EH   (Newton-Schulz)
  OA_T3,      // T3 = C X3 (EG)             -> EX
  OA_A,       // A = X3^T T3                -> EA, and B <- X3
};

__global__ void __launch_bounds__(kFW * 32) k_oa_gemm(Search* S, TileMap tm, int op) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (!mixed_route_due(s)) return;
  const int n = s.n;
  const long long L = s.ldn;
  const double* C = s.C;
  switch (op) {
    case OA_W0: {
      const double* B = s.B;
      double* TT = s.EG;
      gemm_flat_f64<1>(n, t, [=] __device__(int i, int k) { return C[i + L * k]; },
                       [=] __device__(int, int k, int j) { return B[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) { TT[j + L * i] = v; });
      break;
    }
    case OA_W1: {
      const double* TT = s.EG;
      const double* B = s.B;
      double* A = s.EH;
      gemm_flat_f64<1, true>(n, t, [=] __device__(int i, int k) { return TT[i + L * k]; },
                       [=] __device__(int, int k, int j) { return B[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) { A[i + L * j] = v; });
      break;
    }
    case OA_X0: {
      const double* B = s.B;
      const double* V = s.EG;
      double* X = s.ET;
      double* XT = s.EX;
      gemm_flat_f64<1>(n, t, [=] __device__(int i, int k) { return B[i + L * k]; },
                       [=] __device__(int, int k, int j) { return V[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) {
                         X[i + L * j] = v;
                         XT[j + L * i] = v;
                       });
      break;
    }
    case OA_T0:
    case OA_T1:
    case OA_T3: {
      const double* X = op == OA_T0 ? s.ET : s.EG;
      double* T = op == OA_T3 ? s.EX : s.EA;
      gemm_flat_f64<1>(n, t, [=] __device__(int i, int k) { return C[i + L * k]; },
                       [=] __device__(int, int k, int j) { return X[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) { T[i + L * j] = v; });
      break;
    }
    case OA_SG0:
    case OA_SG1: {
      const double* XT = op == OA_SG0 ? s.EX : s.EH;
      const double* X = op == OA_SG0 ? s.ET : s.EG;
      const double* T = s.EA;
      double* So = op == OA_SG0 ? s.EG : s.ET;
      double* Go = op == OA_SG0 ? s.EH : s.EX;
      double* lam = s.D;  // scratch until the Jacobi writes D
      gemm_flat_f64<2, true>(n, t, [=] __device__(int i, int k) { return XT[i + L * k]; },
                       [=] __device__(int a, int k, int j) { return a == 0 ? T[k + L * j] : X[k + L * j]; },
                       [=] __device__(int i, int j, double sv, double gv) {
                         So[i + L * j] = sv;
                         Go[i + L * j] = gv;
                         if (i == j) lam[i] = sv / gv;
                       });
      break;
    }
    case OA_U0:
    case OA_U1: {
      const double* X = op == OA_U0 ? s.ET : s.EG;
      const double* E = s.EA;
      double* Xo = op == OA_U0 ? s.EG : s.B;
      double* XTo = op == OA_U0 ? s.EH : s.ET;
      gemm_flat_f64<1>(n, t, [=] __device__(int i, int k) { return X[i + L * k]; },
                       [=] __device__(int, int k, int j) { return E[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) {
                         const double x = X[i + L * j] + v;
                         Xo[i + L * j] = x;
                         XTo[j + L * i] = x;
                       });
      break;
    }
    case OA_G2: {
      const double* XT = s.ET;
      const double* X = s.B;
      double* M = s.EX;
      gemm_flat_f64<1, true>(n, t, [=] __device__(int i, int k) { return XT[i + L * k]; },
                       [=] __device__(int, int k, int j) { return X[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) {
                         M[i + L * j] = 0.5 * ((i == j ? 1.0 : 0.0) - v);
                       });
      break;
    }
    case OA_N2: {
      const double* X = s.B;
      const double* M = s.EX;
      double* Xo = s.EG;
      double* XTo = s.EH;
      gemm_flat_f64<1>(n, t, [=] __device__(int i, int k) { return X[i + L * k]; },
                       [=] __device__(int, int k, int j) { return M[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) {
                         const double x = X[i + L * j] + v;
                         Xo[i + L * j] = x;
                         XTo[j + L * i] = x;
                       });
      break;
    }
    case OA_A: {
      const double* XT = s.EH;
      const double* X = s.EG;
      const double* T = s.EX;
      double* A = s.EA;
      double* B = s.B;
      gemm_flat_f64<1, true>(n, t, [=] __device__(int i, int k) { return XT[i + L * k]; },
                       [=] __device__(int, int k, int j) { return T[k + L * j]; },
                       [=] __device__(int i, int j, double v, double) {
                         A[i + L * j] = v;
                         B[i + L * j] = X[i + L * j];
                       });
      break;
    }
  }
}

// E of one refinement step from S, G and lambda (elementwise, same output
// order as the products). A pair is corrected to first order only when both
// of its corrections stay below 2^-10; otherwise both entries only get the
// orthogonality half -g_ij / 2. The bound keeps the second-order loss of
// orthogonality of a step, sum_k |e_ki e_kj| <= n 2^-20, small enough that the
// second step and the Newton-Schulz step bring X^T X to I within rounding
// (1.5 (n 2^-20)^4 << eps64 for n <= 160; at larger n only near neighbours in
// the spectrum reach the bound, and what the refinement leaves goes to the
// cleanup Jacobi).
constexpr double kOaSep = 0x1p-10;
__global__ void __launch_bounds__(kFW * 32) k_oa_e(Search* S, TileMap tm, int step) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (!mixed_route_due(s)) return;
  const int n = s.n;
  const long long L = s.ldn;
  const double* Sm = step == 0 ? s.EG : s.ET;
  const double* Gm = step == 0 ? s.EH : s.EX;
  const double* lam = s.D;  // lambda_i = s_ii / g_ii from the product's epilogue
  double* E = s.EA;
  const int base = t * kFO + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kFP; ++u) {
    const int o = base + kFW * 32 * u;
    if (o >= n * n) break;
    const int i = o % n, j = o / n;
    const double gij = Gm[i + L * j];
    double e;
    if (i == j) {
      e = 0.5 * (1.0 - gij);
    } else {
      // the test is symmetric in (i, j), so e_ij + e_ji = -g_ij in both branches
      const double li = lam[i], lj = lam[j];
      const double num = Sm[i + L * j] - lj * gij, num_t = Sm[j + L * i] - li * gij;
      const double den = lj - li, lim = kOaSep * fabs(den);
      e = (fabs(num) <= lim && fabs(num_t) <= lim) ? num / den : -0.5 * gij;
    }
    E[i + L * j] = e;
  }
}

// FP32 cyclic Jacobi on A32 (from EH, symmetrised, shifted and scaled on
// load). Rotations below FP32 resolution are skipped: a pair turns only when
// a_pq^2 > 1e-12 |a_pp a_qq| and |a_pq| > 16 eps32 max|a_ii|.
// A step is bound by its instruction count, so the matrix moves with the
// round-robin ring instead of being addressed through it. Position (k, x)
// is role x (a = 0: the pair's p, b = 1: its q) of pair k; at step r it
// holds element p(r, k) or q(r, k). From step r to r + 1 the ring turns one
// place: (k, a) -> (k - 1, a) for k >= 1, (0, a) -> (1, b), (k, b) ->
// (k + 1, b) for 1 <= k <= P - 2, (P - 1, b) -> (P - 1, a), (0, b) stays.
// The entry between positions (K, x) and (L, y), K < L, is kept in plane
// 2x + y at K P + L; a diagonal block (K, K) keeps a_aa, a_ab, a_bb in planes
// 0, 1, 3 at K P + K. A step reads each off-diagonal block of one buffer,
// rotates it (two-sided, 16 FMAs), and writes its four entries to their
// positions of the next step in the other buffer: all addresses are fixed
// for the whole decomposition and held in registers, and consecutive lanes
// (consecutive L) read and write consecutive words of each plane.
// Further:
//  - A32 is scaled by a power of two so that max|a_ij| <= 1: the scaling is
//    exact, leaves the eigenvectors alone, and keeps the squares of the
//    rotation test and of the angle away from overflow (and, for any spread
//    FP32 can resolve, from underflow);
//  - the rotation (Golub & Van Loan §8.5, t the smaller root of
//    t^2 + 2 theta t - 1 = 0 with theta = (a_qq - a_pp) / (2 a_pq)) is
//    taken as t = sign(theta) 2 |a_pq| / (|d| + sqrt(d^2 + 4 a_pq^2)),
//    d = a_qq - a_pp: one square root and one division, both the fast
//    approximations; c = 1 / sqrt(1 + t^2) is rsqrtf plus one Newton step,
//    s = t c. Any t gives an orthogonal (c, s); its last-bit error only
//    leaves a_pq at FP32 rounding level, which the FP64 refinement removes;
//  - the pivot of next-step pair k lands in the diagonal block (k, k) from
//    exactly one block of the current step: (0, 1) for k = 0, (0, 2) for
//    k = 1, (k - 1, k + 1) for 2 <= k <= P - 2, (P - 2, P - 1) for k = P - 1.
//    The thread owning it forms the next rotation right after its own update
//    (the diagonal entries it needs were finished in the step before) and
//    writes the next diagonal block: one barrier per step. These P role
//    blocks come first in the thread list, so the rotation arithmetic stays
//    in the first warps, and their threads own no other block;
//  - a step without rotations still turns the ring (its blocks only move);
//  - with n odd the padding element N - 1 is the fixed (0, b): pair 0 never
//    rotates and the padding row and column stay exactly zero;
//  - a pair's step record is (c, s); (1, 0) when it does not rotate.
// The eigenvectors are not formed here: each step that rotates anything
// appends its (c, s) table to the rotation log, and k_jlog_apply replays the
// log on the rows of V32 = I across the GPU.
constexpr float kJ32Tol2 = kJ32Tol * kJ32Tol;
__device__ __forceinline__ bool j32_rotates(float app, float aqq, float apq, float floor_abs) {
  return fabsf(apq) > floor_abs && apq * apq > kJ32Tol2 * fabsf(app * aqq);
}

// (c, s, t) of the rotation that annihilates a_pq (a_pq passed j32_rotates,
// so a_pq^2 > 0 and the root's argument is positive)
__device__ __forceinline__ void j32_rotation(float app, float aqq, float apq, float& c, float& s, float& t) {
  const float d = aqq - app;
  const float x = fmaf(d, d, 4.f * apq * apq);
  const float h = x * rsqrtf(x);  // sqrt(d^2 + 4 a_pq^2)
  const float mag = __fdividef(2.f * fabsf(apq), fabsf(d) + h);
  // sign(theta), with theta = +-0 counted as positive
  t = (d == 0.f || ((d > 0.f) == (apq > 0.f))) ? mag : -mag;
  const float u = fmaf(t, t, 1.f);
  float y = rsqrtf(u);
  y = y * fmaf(-0.5f * u * y, y, 1.5f);  // Newton step for 1 / sqrt(u)
  c = y;
  s = t * y;
}

// ring position (K, x) at step r + 1 of the position (K, x) at step r
__device__ __forceinline__ void ring_next(int K, int x, int P, int& Kn, int& xn) {
  if (x == 0) {
    Kn = K >= 1 ? K - 1 : 1;
    xn = K >= 1 ? 0 : 1;
  } else {
    Kn = (K == 0) ? 0 : (K == P - 1 ? P - 1 : K + 1);
    xn = (K == P - 1) ? 0 : 1;
  }
}

// offset (plane * P^2 + slot) of the entry between positions (K, x), (L, y)
__device__ __forceinline__ int ring_offset(int K, int x, int L, int y, int P) {
  const int PP = P * P;
  if (K < L) return (2 * x + y) * PP + K * P + L;
  if (K > L) return (2 * y + x) * PP + L * P + K;
  return (x == y ? 3 * x : 1) * PP + K * P + K;
}

// off-diagonal 2 x 2 blocks per thread at the largest size: one for every
// thread, then the rest of P (P - 1) / 2 over the kJ32NT - P threads that
// form no rotation
constexpr int kJ32Blocks =
    1 + ((kE32Max / 2) * (kE32Max / 2 - 1) / 2 - kJ32NT + (kJ32NT - kE32Max / 2) - 1) / (kJ32NT - kE32Max / 2);

__global__ void __launch_bounds__(kJ32NT, 1) k_jacobi32(Search* S, int s0) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ float sh_amax;
  Search& s = S[s0 + blockIdx.x];
  if (!small_route_due(s)) return;
  constexpr int NW = kJ32NT / 32;
  const int n = s.n, N = n + (n & 1), P = N / 2, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int PP = P * P;
  const int nblk = P * (P - 1) / 2;
  const bool pad = n & 1;  // pair 0 holds the padding element and never rotates
  float2* rec = reinterpret_cast<float2*>(fsm);  // 2 x P step records (c, s)
  float* buf = fsm + 4 * P;                       // 2 buffers x 4 planes x P^2
  // A32 = 2^-k (B^T C B - c I) rounded to FP32, with c the mean eigenvalue
  // (the trace over n, in FP64) and 2^k the power of two at or above
  // max a_ii. B^T C B is positive semi-definite, so |a_ij| <= max a_ii and
  // |a_ii - c| <= max a_ii: every entry of A32 is at most one in magnitude.
  // The shift leaves the eigenvectors alone and lets FP32 resolve the spread
  // of the spectrum around c, which is where nearly equal eigenvalues of an
  // early descent (C close to a multiple of I) live. EH is exactly symmetric
  // (the product writes both triangles), so it is read once, a warp per
  // column with the column's loads issued together, each entry stored at
  // its ring position of step 0: element 0 at (0, a), N - 1 at (0, b),
  // 1 <= e <= P - 1 at (e, a), P <= e <= N - 2 at (N - 1 - e, b).
  const long long L = s.ldn;
  const double* A64 = s.EH;
  double tr = 0.0, dmax = 0.0;
  for (int i = tid; i < n; i += kJ32NT) {
    const double d = A64[i + L * i];
    tr += d;
    dmax = fmax(dmax, fabs(d));
  }
  __shared__ double shs[kJ32NT / 32];
  const double c = block_sum<kJ32NT>(tr, shs) / n;
  dmax = block_max<kJ32NT>(dmax, shs);
  int ex = 0;
  if (dmax > 0.0) frexp(dmax, &ex);  // dmax = m 2^ex, m in [0.5, 1)
  const double scale = ldexp(1.0, -ex);
  const int M = N - 1;
  auto pos0 = [=](int e, int& K, int& x) {
    if (e == 0) { K = 0; x = 0; }
    else if (e == M) { K = 0; x = 1; }
    else if (e <= P - 1) { K = e; x = 0; }
    else { K = M - e; x = 1; }
  };
  constexpr int kRow = (kE32Max + 31) / 32;
  for (int j = warp; j < N; j += NW) {
    double v[kRow];
#pragma unroll
    for (int u = 0; u < kRow; ++u) {
      const int i = lane + 32 * u;
      v[u] = (i < n && j < n) ? A64[i + L * j] : 0.0;
    }
    int Kj, xj;
    pos0(j, Kj, xj);
#pragma unroll
    for (int u = 0; u < kRow; ++u) {
      const int i = lane + 32 * u;
      if (i >= N) continue;
      int Ki, xi;
      pos0(i, Ki, xi);
      // each unordered entry once: the upper block, or the diagonal block's a_aa, a_ab, a_bb
      if (Ki < Kj || (Ki == Kj && xi <= xj))
        buf[ring_offset(Ki, xi, Kj, xj, P)] =
            (i < n && j < n) ? static_cast<float>((v[u] - (i == j ? c : 0.0)) * scale) : 0.f;
    }
  }
  __syncthreads();
  if (warp == 0) {
    float m = 0.f;
    for (int K = lane; K < P; K += 32) m = fmaxf(m, fmaxf(fabsf(buf[K * P + K]), fabsf(buf[3 * PP + K * P + K])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sh_amax = m;
  }
  __syncthreads();
  // Each thread owns the same off-diagonal blocks (K, L), K < L, in every
  // step: entry tid of a list, and entries kJ32NT + (kJ32NT - P)(u - 1) +
  // tid - P for u >= 1 when tid >= P. The list starts with the P role blocks
  // (block k holds the pivot of next-step pair k), then the others row by row
  // (K ascending, L ascending). bKL: K | L << 8 (-1: none); bdst: the four
  // entries' next offsets, (a, a) | (a, b) << 16 and (b, a) | (b, b) << 16.
  int bKL[kJ32Blocks], bdst[kJ32Blocks][2];
#pragma unroll
  for (int u = 0; u < kJ32Blocks; ++u) {
    const int k = u == 0 ? tid : (tid >= P ? kJ32NT + (kJ32NT - P) * (u - 1) + tid - P : nblk);
    int K = 0, Lb = 0;
    if (k < P) {
      if (k == 0) { K = 0; Lb = 1; }
      else if (k == 1) { K = 0; Lb = 2; }
      else if (k == P - 1) { K = P - 2; Lb = P - 1; }
      else { K = k - 1; Lb = k + 1; }
    } else if (k < nblk) {
      // the (k - P)-th block that holds no pivot, row by row: row K has
      // P - 1 - K blocks, of which (K, K + 2), (0, 1) and (P - 2, P - 1) hold one
      int j = k - P;
      for (;;) {
        const int cnt = (P - 1 - K) - (K + 2 <= P - 1) - (K == 0) - (K == P - 2);
        if (j < cnt) break;
        j -= cnt;
        ++K;
      }
      for (Lb = K + 1;; ++Lb) {
        const bool role = (K == 0 && Lb == 1) || (Lb == K + 2) || (K == P - 2 && Lb == P - 1);
        if (role) continue;
        if (j == 0) break;
        --j;
      }
    }
    bKL[u] = k < nblk ? K | (Lb << 8) : -1;
    int d[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int Kn, xn, Ln, yn;
      ring_next(K, e >> 1, P, Kn, xn);
      ring_next(Lb, e & 1, P, Ln, yn);
      d[e] = ring_offset(Kn, xn, Ln, yn, P);
    }
    bdst[u][0] = d[0] | (d[1] << 16);
    bdst[u][1] = d[2] | (d[3] << 16);
  }
  // role of thread tid < P (its block is the list's entry tid): the entry
  // holding the pivot of next pair k = tid (0: (a, a), 2: (b, a), 3: (b, b)),
  // the current offsets of that pair's two diagonal entries, and the next
  // offset of the current diagonal block k's off-diagonal entry
  int r_ent = 0, r_srcA = 0, r_srcB = 0, r_move = 0;
  if (tid < P) {
    const int k = tid;
    r_ent = k == 1 ? 0 : (k == P - 1 ? 3 : 2);
    r_srcA = k <= P - 2 ? ring_offset(k + 1, 0, k + 1, 0, P) : ring_offset(P - 1, 1, P - 1, 1, P);
    r_srcB = k >= 2 ? ring_offset(k - 1, 1, k - 1, 1, P) : ring_offset(0, k == 1 ? 0 : 1, 0, k == 1 ? 0 : 1, P);
    int Ka, xa, Kb, xb;
    ring_next(k, 0, P, Ka, xa);
    ring_next(k, 1, P, Kb, xb);
    r_move = ring_offset(Ka, xa, Kb, xb, P);
  }
  // below 16 eps32 max|a_ii| an off-diagonal entry is FP32 rounding noise
  const float floor_abs = 16.f * 1.1920929e-7f * sh_amax;
  const int cap = jlog_steps_cap(n);
  float2* jlog = reinterpret_cast<float2*>(s.jlog);
  int logged = 0;
  // The rotation of pair k of step rn from its 2 x 2 diagonal block: the
  // new diagonal entries, the step record, and the log entry (at the index
  // the step gets if it rotates anything: later rotating steps overwrite the
  // entries of a quiet one). Returns whether it rotates; apq becomes zero then.
  auto rotate_pair = [&](int rn, int k, float& app, float& aqq, float& apq, float2* recn) -> int {
    float cr = 1.f, sr = 0.f;
    int act = 0;
    if (!(pad && k == 0) && j32_rotates(app, aqq, apq, floor_abs)) {
      float tn;
      j32_rotation(app, aqq, apq, cr, sr, tn);
      app -= tn * apq;
      aqq += tn * apq;
      apq = 0.f;
      act = 1;
    }
    recn[k] = make_float2(cr, sr);
    if (logged < cap) {
      jlog[static_cast<size_t>(logged) * P + k] = make_float2(cr, sr);
      if (k == 0) s.jlog_r[logged] = rn;
    }
    return act;
  };
  // step 0: the rotations from the diagonal blocks of buffer 0
  int act0 = 0;
  if (tid < P) {
    float app = buf[tid * P + tid], aqq = buf[3 * PP + tid * P + tid], apq = buf[PP + tid * P + tid];
    act0 = rotate_pair(0, tid, app, aqq, apq, rec);
    buf[tid * P + tid] = app;
    buf[3 * PP + tid * P + tid] = aqq;
    buf[PP + tid * P + tid] = apq;
  }
  int nact = __syncthreads_count(act0);
  int cur = 0, r = 0, sweep = 0, quiet = 0;
  bool converged = false;
  while (true) {
    // step r: its rotations are in the records of buffer cur (diagonal blocks applied)
    const float* bc = buf + cur * 4 * PP;
    if (nact == 0) {
      // a quiet step: if no off-diagonal entry passes the test any more, the
      // remaining quiet steps of the window would change nothing
      ++quiet;
      if (quiet == 1 || (quiet & 15) == 0) {
        int pend = 0;
        for (int e = tid; e < PP && !pend; e += kJ32NT) {
          const int K = e / P, Lb = e % P;
          if (K > Lb) continue;
          const float aK = bc[K * P + K], bK = bc[3 * PP + K * P + K];
          if (K == Lb) {
            pend |= j32_rotates(aK, bK, bc[PP + e], floor_abs);
          } else {
            const float aL = bc[Lb * P + Lb], bL = bc[3 * PP + Lb * P + Lb];
            pend |= j32_rotates(aK, aL, bc[e], floor_abs) | j32_rotates(aK, bL, bc[PP + e], floor_abs) |
                    j32_rotates(bK, aL, bc[2 * PP + e], floor_abs) | j32_rotates(bK, bL, bc[3 * PP + e], floor_abs);
          }
        }
        if (!__syncthreads_or(pend)) quiet = M;
      }
      if (quiet >= M) {
        converged = true;
        break;  // uniform: the counts come from block barriers
      }
    } else {
      quiet = 0;
      ++logged;  // its log entries were written with its rotations
    }
    const int rn = (r + 1 == M) ? 0 : r + 1;
    if (rn == 0 && ++sweep == kJ32MaxSweeps) break;
    // A <- J^T A J on the thread's blocks, each entry written to its position
    // of step rn in the other buffer; the role threads form the rotations of
    // step rn and write the next diagonal blocks
    float* bn = buf + (cur ^ 1) * 4 * PP;
    const float2* rc = rec + cur * P;
    float2* rnx = rec + (cur ^ 1) * P;
    int act = 0;
#pragma unroll
    for (int u = 0; u < kJ32Blocks; ++u) {
      if (bKL[u] < 0) continue;
      const int K = bKL[u] & 0xff, Lb = bKL[u] >> 8;
      const int o = K * P + Lb;
      float x[4] = {bc[o], bc[PP + o], bc[2 * PP + o], bc[3 * PP + o]};
      const float2 gK = rc[K], gL = rc[Lb];
      if (gK.y != 0.f || gL.y != 0.f) {
        const float cP = gK.x, sP = gK.y, cQ = gL.x, sQ = gL.y;
        const float y00 = x[0] * cQ - x[1] * sQ, y01 = x[0] * sQ + x[1] * cQ;
        const float y10 = x[2] * cQ - x[3] * sQ, y11 = x[2] * sQ + x[3] * cQ;
        x[0] = cP * y00 - sP * y10;
        x[1] = cP * y01 - sP * y11;
        x[2] = sP * y00 + cP * y10;
        x[3] = sP * y01 + cP * y11;
      }
      if (u == 0 && tid < P) {
        const int k = tid;
        float app = bc[r_srcA], aqq = bc[r_srcB];
        float apq = r_ent == 0 ? x[0] : (r_ent == 2 ? x[2] : x[3]);
        act = rotate_pair(rn, k, app, aqq, apq, rnx);
        if (r_ent == 0) x[0] = apq;
        else if (r_ent == 2) x[2] = apq;
        else x[3] = apq;
        bn[k * P + k] = app;
        bn[3 * PP + k * P + k] = aqq;
        bn[r_move] = bc[PP + k * P + k];  // the current diagonal block's a_ab moves on
      }
      bn[bdst[u][0] & 0xffff] = x[0];
      bn[bdst[u][0] >> 16] = x[1];
      bn[bdst[u][1] & 0xffff] = x[2];
      bn[bdst[u][1] >> 16] = x[3];
    }
    nact = __syncthreads_count(act);
    cur ^= 1;
    r = rn;
  }
  if (tid == 0) {
    s.jlog_steps = logged;
    s.eig_sweeps32 += converged ? sweep + 1 : sweep;
  }
}

int jacobi32_smem_bytes(int n) {
  const int N = n + (n & 1), P = N / 2;
  return 2 * P * 8 + 2 * 4 * P * P * 4;
}

// V32 from the rotation log: row i of V32 = e_i^T J_1 J_2 ... J_T, and the
// rows are independent, so one warp replays the log on one row, held in
// registers. At step r lane l of slot u holds, for the round-robin pair
// pi = l + 32 u, a_pi = v[p(r, pi)] and b_pi = v[q(r, pi)]; the rotation of
// the pair is then local to the lane. From step r to r + 1 (mod N - 1) the
// ring a_0, a_1, ..., a_{P-1}, b_{P-1}, ..., b_1 moves one place (b_0 = v[N - 1]
// stays): a_pi <- a_{pi+1}, b_pi <- b_{pi-1}, a_{P-1} <- b_{P-1}, b_1 <- a_0,
// two shuffles per slot plus one broadcast. Steps the Jacobi did not log (no
// rotation) are extra moves of the ring.
// The log streams through shared memory in chunks of whole steps, up to
// kLogChunkMax (c, s) entries (a chunk is contiguous in the log): the CTA's
// loads of chunk c + 1 are in flight while its warps apply chunk c. The CTA's
// kLogRows rows leave as FP64 into EG (V32 is read from there by X0 = B V32),
// 8 consecutive rows of a column per store group.
constexpr int kLogRows = 8;
constexpr int kLogNT = kLogRows * 32;
constexpr int kLogChunkMax = 2048;  // (c, s) entries per chunk
constexpr int kLogLoads = kLogChunkMax / kLogNT;
constexpr int kLogStepsMax = kLogChunkMax / 16;  // steps per chunk at the smallest P (n > 32)
static_assert(kJacobiSmallN >= 32, "the refined route starts above n = 32: P >= 17");

// round-robin pair pi of step r (N - 1 = M): (r, M) for pi = 0, else
// ((r + pi) mod M, (r - pi) mod M), as in k_jacobi32
__device__ __forceinline__ void rr_pair(int r, int pi, int M, int& p, int& q) {
  p = r + pi;
  q = r - pi;
  if (p >= M) p -= M;
  if (q < 0) q += M;
  if (pi == 0) q = M;
}

template <int PL>  // slots per lane: P <= 32 PL
__device__ __forceinline__ void jlog_replay(const Search& s, float* v, float2 (*lcs)[kLogChunkMax],
                                            int (*lr)[kLogStepsMax]) {
  const int n = s.n, N = n + (n & 1), P = N / 2, M = N - 1;
  const int tid = threadIdx.x, lane = tid & 31;
  const float2* jlog = reinterpret_cast<const float2*>(s.jlog);
  const int T = s.jlog_steps;
  const int K = kLogChunkMax / P;  // steps per chunk (<= kLogStepsMax)
  const int nch = ceil_div(T, K);
  float2 stage[kLogLoads];
  int rstage = 0;
  auto load = [&](int c) {  // chunk c into registers: entries [c K P, min(T, (c + 1) K) P)
    const int t0 = c * K, cnt = min(K, T - t0);
    const float2* src = jlog + static_cast<size_t>(t0) * P;
#pragma unroll
    for (int u = 0; u < kLogLoads; ++u) {
      const int e = tid + u * kLogNT;
      if (e < cnt * P) stage[u] = __ldg(src + e);
    }
    if (tid < cnt) rstage = __ldg(s.jlog_r + t0 + tid);
  };
  auto store = [&](int c, int buf) {
    const int cnt = min(K, T - c * K);
#pragma unroll
    for (int u = 0; u < kLogLoads; ++u) {
      const int e = tid + u * kLogNT;
      if (e < cnt * P) lcs[buf][e] = stage[u];
    }
    if (tid < cnt) lr[buf][tid] = rstage;
  };
  if (nch == 0) return;  // no rotation: the row stays e_i
  load(0);
  store(0, 0);
  __syncthreads();
  // the ring at the first logged step
  int r = lr[0][0];
  float a[PL], b[PL];
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int pi = lane + 32 * u;
    a[u] = b[u] = 0.f;
    if (pi < P) {
      int p, q;
      rr_pair(r, pi, M, p, q);
      a[u] = v[p];
      b[u] = v[q];
    }
  }
  auto shift = [&]() {  // step r -> r + 1
    float ra[PL], rb[PL];
#pragma unroll
    for (int u = 0; u < PL; ++u) {
      ra[u] = __shfl_sync(0xffffffffu, a[u], (lane + 1) & 31);
      rb[u] = __shfl_sync(0xffffffffu, b[u], (lane - 1) & 31);
    }
    const float a00 = __shfl_sync(0xffffffffu, a[0], 0);
#pragma unroll
    for (int u = 0; u < PL; ++u) {
      const int pi = lane + 32 * u;
      const float up_next = lane < 31 ? ra[u] : (u + 1 < PL ? ra[u + 1 < PL ? u + 1 : u] : 0.f);
      const float dn_prev = lane > 0 ? rb[u] : (u > 0 ? rb[u > 0 ? u - 1 : 0] : 0.f);
      const float na = pi == P - 1 ? b[u] : up_next;
      const float nb = pi == 0 ? b[u] : (pi == 1 ? a00 : dn_prev);
      a[u] = na;
      b[u] = nb;
    }
  };
  for (int c = 0; c < nch; ++c) {
    const int cur = c & 1;
    if (c + 1 < nch) load(c + 1);  // in flight during the steps of chunk c
    const int cnt = min(K, T - c * K);
    const float2* cs = lcs[cur];
    for (int k = 0; k < cnt; ++k, cs += P) {
      const int rk = lr[cur][k];
      int moves = rk - r;  // unlogged steps between the two logged ones, plus one
      if (moves < 0) moves += M;
      for (int j = 0; j < moves; ++j) shift();
      r = rk;
#pragma unroll
      for (int u = 0; u < PL; ++u) {
        const int pi = lane + 32 * u;
        if (pi < P) {
          const float2 g = cs[pi];
          const float x = a[u], y = b[u];
          a[u] = g.x * x - g.y * y;
          b[u] = g.y * x + g.x * y;
        }
      }
    }
    // the other buffer was last read in chunk c - 1, before the barrier below it
    if (c + 1 < nch) store(c + 1, cur ^ 1);
    __syncthreads();
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int pi = lane + 32 * u;
    if (pi < P) {
      int p, q;
      rr_pair(r, pi, M, p, q);
      v[p] = a[u];
      v[q] = b[u];
    }
  }
}

__global__ void __launch_bounds__(kLogNT) k_jlog_apply(Search* S, int s0) {
  __shared__ float vrow[kLogRows][kE32Max + 1];
  __shared__ float2 lcs[2][kLogChunkMax];
  __shared__ int lr[2][kLogStepsMax];
  const Search& s = S[s0 + blockIdx.y];
  if (!small_route_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2;
  const int i0 = blockIdx.x * kLogRows;
  if (i0 >= n) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, i = i0 + warp;
  float* v = vrow[warp];
  for (int j = lane; j < N; j += 32) v[j] = (j == i) ? 1.f : 0.f;  // rows past n stay zero
  __syncwarp();
  if (P <= 32)
    jlog_replay<1>(s, v, lcs, lr);
  else if (P <= 64)
    jlog_replay<2>(s, v, lcs, lr);
  else
    jlog_replay<3>(s, v, lcs, lr);
  __syncthreads();
  const long long L = s.ldn;
  const int rows = min(kLogRows, n - i0);
  for (int e = tid; e < kLogRows * n; e += kLogNT) {
    const int ii = e % kLogRows, j = e / kLogRows;
    if (ii < rows) s.EG[(i0 + ii) + L * j] = static_cast<double>(vrow[ii][j]);
  }
}

// Targeted rotations before the cyclic cleanup. After the refinement only a
// handful of pairs of nearly equal eigenvalues can still pass the FP64 Jacobi
// test, and the cyclic order would need up to n - 1 mostly empty steps to
// reach them. Here one CTA per search works on A (EA) and V (B) in global
// memory for up to kRoundsMax rounds: find every pair that passes the test the
// cleanup uses (same threshold, same rounding floor), take a disjoint set of
// the largest ones, apply their exact rotations (columns of A, then rows, then
// the 2 x 2 blocks set exactly, then V's columns). A round with nothing
// pending ends the kernel; more than kRoundsList pending pairs leaves them all
// to the cyclic sweeps, which remain the correctness backstop either way.
// A lives in shared memory for the whole kernel (leading dimension n + 1, up to
// 161 x 160 doubles) and goes back to EA only if a rotation was applied: a
// round then costs shared-memory passes instead of a scan of A through L2.
// Mixed-precision handles only: the FP64 handles' stricter floor leaves tens
// of noise-level pairs, which the cluster's 8 SMs rotate faster than one CTA.
constexpr int kRoundsNT = 512;
constexpr int kRoundsMax = 16;
constexpr int kRoundsList = 512;
constexpr int kRoundsPick = kEigMixedMaxN / 2;  // every disjoint pending pair
constexpr double kRoundsTol = 1e-14;  // the cyclic FP64 Jacobi's relative threshold

__global__ void __launch_bounds__(kRoundsNT) k_pair_rounds(Search* S, int s0) {
  extern __shared__ double As[];  // A, leading dimension n + 1
  __shared__ int cnt, npick;
  // candidate keys: ~(top 48 bits of |a_pq|) << 16 | p << 8 | q, so that an
  // ascending sort gives the largest entries first and ties by index: the
  // order, and so the rotations, do not depend on thread timing
  __shared__ unsigned long long ckey[kRoundsList];
  __shared__ int pp[kRoundsPick], pq[kRoundsPick];
  __shared__ double pc[kRoundsPick], ps[kRoundsPick], pt[kRoundsPick];
  __shared__ double papp[kRoundsPick], paqq[kRoundsPick], papq[kRoundsPick];
  __shared__ double shr[kRoundsNT / 32];
  Search& s = S[s0 + blockIdx.x];
  if (!small_route_due(s) || !s.mixed) return;
  const int n = s.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long L = s.ldn;
  double* Ag = s.EA;
  double* V = s.B;
  const int la = n + 1;
  constexpr int kRow = (kEigMixedMaxN + 31) / 32;  // rows per lane of a column
  // a warp per column, its loads issued together (one L2 round trip per column)
  for (int j = warp; j < n; j += kRoundsNT / 32) {
    double x[kRow];
#pragma unroll
    for (int u = 0; u < kRow; ++u) {
      const int i = lane + 32 * u;
      x[u] = i < n ? Ag[i + L * j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kRow; ++u) {
      const int i = lane + 32 * u;
      if (i < n) As[i + la * j] = x[u];
    }
  }
  __syncthreads();
  double* A = As;
  double am = 0.0;
  for (int i = tid; i < n; i += kRoundsNT) am = fmax(am, fabs(A[i + la * i]));
  const double amax = block_max<kRoundsNT>(am, shr);
  const double floor_abs = 4.0 * n * 0x1p-53 * amax;  // the cleanup's floor on mixed handles
  const long long floor_bits = __double_as_longlong(floor_abs);
  long long rot_total = 0;
  for (int round = 0; round < kRoundsMax; ++round) {
    if (tid == 0) cnt = 0;
    __syncthreads();
    // every pair p < q; entries at or below the floor are rejected on their
    // bit pattern (non-negative doubles order as integers)
    for (int q = warp; q < n; q += kRoundsNT / 32) {
      const long long* col = reinterpret_cast<const long long*>(A + la * q);
      long long bits[kRow];  // |a_pq| as integers, loaded together
#pragma unroll
      for (int u = 0; u < kRow; ++u) {
        const int p = lane + 32 * u;
        bits[u] = p < q ? (col[p] & 0x7fffffffffffffffll) : 0;
      }
#pragma unroll
      for (int u = 0; u < kRow; ++u) {
        if (bits[u] <= floor_bits) continue;  // the FP64 test only above the floor
        const int p = lane + 32 * u;
        const double apq = A[p + la * q];
        if (!jacobi_rotates(A[p + la * p], A[q + la * q], apq, kRoundsTol * kRoundsTol, floor_abs)) continue;
        const int k = atomicAdd(&cnt, 1);
        if (k < kRoundsList) {
          const unsigned long long mag = static_cast<unsigned long long>(bits[u]);
          ckey[k] = (~(mag >> 16) << 16) | (static_cast<unsigned>(p) << 8) | static_cast<unsigned>(q);
        }
      }
    }
    __syncthreads();
    const int c = cnt;
    if (c == 0 || c > kRoundsList) break;  // done, or too many: the cyclic sweeps take them
    // bitonic sort of the candidate keys (padded to a power of two)
    int cap = 1;
    while (cap < c) cap <<= 1;
    for (int i = c + tid; i < cap; i += kRoundsNT) ckey[i] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= cap; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = tid; i < cap; i += kRoundsNT) {
          const int j = i ^ stride;
          if (j > i) {
            const bool up = (i & size) == 0;
            const unsigned long long a = ckey[i], b = ckey[j];
            if ((a > b) == up) {
              ckey[i] = b;
              ckey[j] = a;
            }
          }
        }
        __syncthreads();
      }
    if (tid == 0) {  // greedy disjoint set in key order
      unsigned used[(kEigMixedMaxN + 31) / 32] = {0};
      int m = 0;
      for (int j = 0; j < c && m < kRoundsPick; ++j) {
        const int p = static_cast<int>((ckey[j] >> 8) & 0xff), q = static_cast<int>(ckey[j] & 0xff);
        if ((used[p >> 5] >> (p & 31)) & 1u || (used[q >> 5] >> (q & 31)) & 1u) continue;
        used[p >> 5] |= 1u << (p & 31);
        used[q >> 5] |= 1u << (q & 31);
        pp[m] = p;
        pq[m] = q;
        ++m;
      }
      npick = m;
    }
    __syncthreads();
    const int m = npick;
    if (tid < m) {
      const int p = pp[tid], q = pq[tid];
      const double app = A[p + la * p], aqq = A[q + la * q], apq = A[p + la * q];
      double t, cc, sn;
      jacobi_rotation(app, aqq, apq, t, cc, sn);
      pc[tid] = cc;
      ps[tid] = sn;
      pt[tid] = t;
      papp[tid] = app;
      paqq[tid] = aqq;
      papq[tid] = apq;
    }
    __syncthreads();
    for (int e = tid; e < m * n; e += kRoundsNT) {  // A <- A J: columns p, q
      const int k = e / n, r = e % n;
      double* ap = A + la * pp[k];
      double* aq = A + la * pq[k];
      const double x = ap[r], y = aq[r];
      ap[r] = pc[k] * x - ps[k] * y;
      aq[r] = ps[k] * x + pc[k] * y;
    }
    __syncthreads();
    for (int e = tid; e < m * n; e += kRoundsNT) {  // A <- J^T A: rows p, q
      const int k = e / n, col = e % n;
      const int o = la * col;
      const double x = A[pp[k] + o], y = A[pq[k] + o];
      A[pp[k] + o] = pc[k] * x - ps[k] * y;
      A[pq[k] + o] = ps[k] * x + pc[k] * y;
    }
    __syncthreads();
    if (tid < m) {  // exact 2 x 2 diagonal block
      const int p = pp[tid], q = pq[tid];
      A[p + la * p] = papp[tid] - pt[tid] * papq[tid];
      A[q + la * q] = paqq[tid] + pt[tid] * papq[tid];
      A[p + la * q] = 0.0;
      A[q + la * p] = 0.0;
    }
    for (int e = tid; e < m * n; e += kRoundsNT) {  // V <- V J
      const int k = e / n, r = e % n;
      double* vp = V + L * pp[k];
      double* vq = V + L * pq[k];
      const double x = vp[r], y = vq[r];
      vp[r] = pc[k] * x - ps[k] * y;
      vq[r] = ps[k] * x + pc[k] * y;
    }
    rot_total += m;
    __syncthreads();
  }
  if (rot_total > 0)  // uniform: every thread counts the same rounds
    for (int j = warp; j < n; j += kRoundsNT / 32)
      for (int i = lane; i < n; i += 32) Ag[i + L * j] = As[i + la * j];
  if (tid == 0) s.eig_rotations += rot_total;
}

int pair_rounds_smem_bytes(int n) { return (n + 1) * n * 8; }


int launch_eig_mixed_head(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st) {
  if (tflat.total <= 0 || s1 <= s0) return 0;
  int nl = 0;
  k_oa_gemm<<<tflat.total, kFW * 32, 0, st>>>(S, tflat, OA_W0);
  k_oa_gemm<<<tsym.total, kFW * 32, 0, st>>>(S, tsym, OA_W1);  // symmetric result: upper triangle only
  nl += 2;
  if (max_n > kJacobiSmallN) {
    const int mn = max_n < kE32Max ? max_n : kE32Max;
    const int bytes = jacobi32_smem_bytes(mn);
    cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    k_jacobi32<<<s1 - s0, kJ32NT, bytes, st>>>(S, s0);
    k_jlog_apply<<<dim3(ceil_div(mn, kLogRows), s1 - s0), kLogRows * 32, 0, st>>>(S, s0);
    nl += 2;
  }
  return nl;
}

int launch_eig_mixed_tail(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st) {
  if (tflat.total <= 0 || s1 <= s0) return 0;
  int nl = 0;
  const int gf = tflat.total, gs = tsym.total;
  auto flat = [&](int op) {  // products with a general result
    k_oa_gemm<<<gf, kFW * 32, 0, st>>>(S, tflat, op);
    ++nl;
  };
  auto sym = [&](int op) {   // products with a symmetric result: upper triangle only
    k_oa_gemm<<<gs, kFW * 32, 0, st>>>(S, tsym, op);
    ++nl;
  };
  flat(OA_X0);
  for (int step = 0; step < 2; ++step) {
    flat(step == 0 ? OA_T0 : OA_T1);
    sym(step == 0 ? OA_SG0 : OA_SG1);
    k_oa_e<<<gf, kFW * 32, 0, st>>>(S, tflat, step);
    ++nl;
    flat(step == 0 ? OA_U0 : OA_U1);
  }
  sym(OA_G2);
  flat(OA_N2);
  flat(OA_T3);
  sym(OA_A);
  const int mn = max_n < kE32Max ? max_n : kE32Max;
  const int rbytes = pair_rounds_smem_bytes(mn);
  cudaFuncSetAttribute(k_pair_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, rbytes);
  k_pair_rounds<<<s1 - s0, kRoundsNT, rbytes, st>>>(S, s0);
  ++nl;
  return nl;
}

int launch_eig_mixed(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st) {
  return launch_eig_mixed_head(S, tflat, tsym, s0, s1, max_n, st) +
         launch_eig_mixed_tail(S, tflat, tsym, s0, s1, max_n, st);
}

}  // namespace cmaes_gb300
