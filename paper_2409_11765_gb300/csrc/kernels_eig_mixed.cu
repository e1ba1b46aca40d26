// kernels_eig_mixed.cu -- mixed-precision preconditioning of the warm-started
// Jacobi eigendecomposition (mixed-precision handles only).
//
// The FP64 Jacobi of kernels_eig.cu / kernels_jacobi_cluster.cu needs about
// seven sweeps per decomposition when C moves a lot between generations, and on
// GB300 every sweep is bound by the FP64 pipe. Here most of those sweeps run in
// FP32 (a 64x faster pipe) and the FP64 Jacobi only finishes the job:
//   1. A32 = B^T C B in FP32 (the warm start, from the previous basis B).
//   2. FP32 cyclic Jacobi on A32 (same round-robin ordering and rotation
//      formula) until the off-diagonal reaches FP32 resolution; V32 collects
//      the rotations (V32 ~ the eigenvectors of A32, orthonormal to ~1e-6).
//   3. W = B V32 in FP64, made orthonormal to FP64 precision by two
//      Newton-Schulz steps W <- W (3 I - W^T W) / 2 (error e -> 1.5 e^2).
//   4. A = W^T C W in FP64 (nearly diagonal), B <- W; the FP64 Jacobi then
//      runs on (A, B) exactly as in the FP64 path and delivers the FP64
//      eigenvalues, eigenvectors and canonical form.
// Every product here is a small dense GEMM on CUDA cores (32 x 32 tiles so that
// n = 100 still spreads over many SMs); the tensor cores are not used because
// step 3 and 4 need FP64 and step 1 feeds a FP32-accurate Jacobi.
#include <cmath>
#include "device_common.cuh"

namespace cmaes_gb300 {

constexpr int kE32Max = 160;            // FP32 Jacobi keeps A32 and V32 in shared memory
constexpr int kJ32NT = 1024;
constexpr float kJ32Tol = 1e-6f;
constexpr int kJ32MaxSweeps = 20;

int eig_mixed_max_n() { return kE32Max; }
int tiles_square32(int n) { const int t = ceil_div(n, 32); return t * t; }

// 32 x 32 output tile, K step 32, 256 threads with 2 x 2 outputs each.
template <typename T>
struct Gemm32Smem {
  T As[32][33];
  T Bs[32][33];
};

template <typename T, class LA, class LB, class EPI>
__device__ __forceinline__ void gemm32_tile(int M, int N, int K, int i0, int j0, const LA& la, const LB& lb,
                                            const EPI& epi, Gemm32Smem<T>& sm) {
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  T acc[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int a = e & 31, b = e >> 5;  // a fastest
      sm.As[b][a] = (i0 + a < M && k0 + b < K) ? la(i0 + a, k0 + b) : T(0);
      sm.Bs[a][b] = (k0 + a < K && j0 + b < N) ? lb(k0 + a, j0 + b) : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const T a0 = sm.As[kk][tr], a1 = sm.As[kk][tr + 16];
      const T b0 = sm.Bs[kk][tc], b1 = sm.Bs[kk][tc + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = i0 + tr + 16 * r, j = j0 + tc + 16 * c;
      if (i < M && j < N) epi(i, j, acc[r][c]);
    }
}

enum EigOp { OP_CB32 = 0, OP_BTT32, OP_BV, OP_WTW, OP_WM, OP_CW, OP_WTT };

// One stage of the preconditioning, over the searches whose decomposition is
// due and that take the mixed route. Scratch: F32a, F32b (n x n floats, ld n),
// ET and EA (FP64 n x n, ld ldn).
__global__ void __launch_bounds__(256) k_eig_stage(Search* S, TileMap tm, int op) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !s.eig_due || !s.mixed || s.n > kE32Max || s.n <= 32) return;
  const int n = s.n, ldn = s.ldn, T = ceil_div(n, 32);
  const int i0 = (t % T) * 32, j0 = (t / T) * 32;
  const long long L = ldn;
  float* f32a = s.F32a;
  float* f32b = s.F32b;
  const double* C = s.C;
  double* B = s.B;
  double* ET = s.ET;
  double* EA = s.EA;
  if (op == OP_CB32 || op == OP_BTT32) {
    __shared__ Gemm32Smem<float> sm;
    if (op == OP_CB32)  // F32b = C B
      gemm32_tile<float>(n, n, n, i0, j0,
                         [=] __device__(int i, int k) { return static_cast<float>(C[i + L * k]); },
                         [=] __device__(int k, int j) { return static_cast<float>(B[k + L * j]); },
                         [=] __device__(int i, int j, float v) { f32b[i + n * j] = v; }, sm);
    else                // F32a = B^T F32b
      gemm32_tile<float>(n, n, n, i0, j0,
                         [=] __device__(int i, int k) { return static_cast<float>(B[k + L * i]); },
                         [=] __device__(int k, int j) { return f32b[k + n * j]; },
                         [=] __device__(int i, int j, float v) { f32a[i + n * j] = v; }, sm);
    return;
  }
  __shared__ Gemm32Smem<double> sm;
  switch (op) {
    case OP_BV:   // ET = B V32 (V32 in F32b)
      gemm32_tile<double>(n, n, n, i0, j0, [=] __device__(int i, int k) { return B[i + L * k]; },
                          [=] __device__(int k, int j) { return static_cast<double>(f32b[k + n * j]); },
                          [=] __device__(int i, int j, double v) { ET[i + L * j] = v; }, sm);
      break;
    case OP_WTW:  // EA = (3 I - W^T W) / 2 with W = ET
      gemm32_tile<double>(n, n, n, i0, j0, [=] __device__(int i, int k) { return ET[k + L * i]; },
                          [=] __device__(int k, int j) { return ET[k + L * j]; },
                          [=] __device__(int i, int j, double v) { EA[i + L * j] = (i == j ? 1.5 : 0.0) - 0.5 * v; },
                          sm);
      break;
    case OP_WM:   // B = W M (W = ET, M = EA); the Newton-Schulz step
      gemm32_tile<double>(n, n, n, i0, j0, [=] __device__(int i, int k) { return ET[i + L * k]; },
                          [=] __device__(int k, int j) { return EA[k + L * j]; },
                          [=] __device__(int i, int j, double v) { B[i + L * j] = v; }, sm);
      break;
    case OP_CW:   // ET = C B
      gemm32_tile<double>(n, n, n, i0, j0, [=] __device__(int i, int k) { return C[i + L * k]; },
                          [=] __device__(int k, int j) { return B[k + L * j]; },
                          [=] __device__(int i, int j, double v) { ET[i + L * j] = v; }, sm);
      break;
    case OP_WTT:  // EA = B^T ET
      gemm32_tile<double>(n, n, n, i0, j0, [=] __device__(int i, int k) { return B[k + L * i]; },
                          [=] __device__(int k, int j) { return ET[k + L * j]; },
                          [=] __device__(int i, int j, double v) { EA[i + L * j] = v; }, sm);
      break;
  }
}

// ET <- B (the second Newton-Schulz step starts from the first one's result).
__global__ void __launch_bounds__(256) k_eig_copy_b(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !s.eig_due || !s.mixed || s.n > kE32Max || s.n <= 32) return;
  const int n = s.n, ldn = s.ldn, T = ceil_div(n, 32);
  const int i0 = (t % T) * 32, j0 = (t / T) * 32;
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int i = i0 + (e & 31), j = j0 + (e >> 5);
    if (i < n && j < n) s.ET[i + static_cast<long long>(ldn) * j] = s.B[i + static_cast<long long>(ldn) * j];
  }
}

// FP32 cyclic Jacobi on A32 (F32a, symmetrised on load) with V32 = I; V32 is
// written to F32b. Rotations below FP32 resolution are skipped: a pair turns
// only when |a_pq| > 1e-6 sqrt|a_pp a_qq| and |a_pq| > 16 eps32 max|a_ii|.
// FP32 arithmetic is cheap here, so a step costs its instruction count: the
// rotation table is packed (p | q << 10 | rotate << 20, (c, s) as float2),
// the upper-triangle 2 x 2 blocks come from a table built once, V <- V J runs
// one warp per pair over the rows, and the rotation count of a step is the
// barrier's own count.
__device__ __forceinline__ bool j32_rotates(float app, float aqq, float apq, float floor_abs) {
  return fabsf(apq) > floor_abs && fabsf(apq) > kJ32Tol * sqrtf(fabsf(app * aqq));
}

__global__ void __launch_bounds__(kJ32NT, 1) k_jacobi32(Search* S, int s0) {
  extern __shared__ float fsm[];
  __shared__ float sh_amax;
  Search& s = S[s0 + blockIdx.x];
  if (s.done || !s.eig_due || !s.mixed || s.n > kE32Max || s.n <= 32) return;
  constexpr int NW = kJ32NT / 32;
  const int n = s.n, N = n + (n & 1), P = N / 2, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int lda = N + 1;
  const int nblk = P * (P + 1) / 2;
  float* A = fsm;
  float* V = A + lda * N;
  float2* rcs = reinterpret_cast<float2*>(V + lda * N);  // N lda even: 8-byte aligned
  float* rt = reinterpret_cast<float*>(rcs + P);
  int* rpq = reinterpret_cast<int*>(rt + P);
  int* blk = rpq + P;  // block b = Qi (Qi + 1) / 2 + Pi, Pi <= Qi: Pi | Qi << 16
  for (int e = tid; e < N * N; e += kJ32NT) {
    const int i = e % N, j = e / N;
    float a = 0.f;
    if (i < n && j < n) a = 0.5f * (s.F32a[i + n * j] + s.F32a[j + n * i]);
    A[i + lda * j] = a;
    V[i + lda * j] = (i == j && i < n) ? 1.f : 0.f;
  }
  for (int Qi = warp; Qi < P; Qi += NW)
    for (int Pi = lane; Pi <= Qi; Pi += 32) blk[Qi * (Qi + 1) / 2 + Pi] = Pi | (Qi << 16);
  __syncthreads();
  if (warp == 0) {
    float m = 0.f;
    for (int i = lane; i < n; i += 32) m = fmaxf(m, fabsf(A[i + lda * i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sh_amax = m;
  }
  __syncthreads();
  // below 16 eps32 max|a_ii| an off-diagonal entry is FP32 rounding noise
  const float floor_abs = 16.f * 1.1920929e-7f * sh_amax;
  const int M = N - 1;
  int quiet = 0, sweep = 0;
  bool converged = false;
  for (; sweep < kJ32MaxSweeps && !converged; ++sweep) {
    for (int r = 0; r < M; ++r) {
      int act = 0;
      if (tid < P) {  // round-robin pair tid of step r (player N - 1 fixed)
        const int p = (tid == 0) ? r : (r + tid) % M;
        const int q = (tid == 0) ? M : (r - tid + M) % M;
        float c = 1.f, sn = 0.f, tn = 0.f;
        if (p < n && q < n) {
          const float app = A[p + lda * p], aqq = A[q + lda * q], apq = A[p + lda * q];
          if (j32_rotates(app, aqq, apq, floor_abs)) {
            const float theta = (aqq - app) / (2.f * apq);
            const float at = fabsf(theta);
            tn = (at > 1e18f) ? 0.5f / theta : (theta >= 0.f ? 1.f : -1.f) / (at + sqrtf(theta * theta + 1.f));
            c = 1.f / sqrtf(tn * tn + 1.f);
            sn = tn * c;
            act = 1;
          }
        }
        rcs[tid] = make_float2(c, sn);
        rt[tid] = tn;
        rpq[tid] = p | (q << 10) | (act << 20);
      }
      const int nact = __syncthreads_count(act);
      if (nact == 0) {
        // a quiet step: if no off-diagonal entry passes the test any more, the
        // remaining quiet steps of the window would change nothing
        ++quiet;
        if (quiet == 1 || (quiet & 15) == 0) {
          int pend = 0;
          for (int Qi = warp; Qi < n && !pend; Qi += NW) {
            const float aqq = A[Qi + lda * Qi];
            for (int Pi = lane; Pi < Qi; Pi += 32)
              pend |= j32_rotates(A[Pi + lda * Pi], aqq, A[Pi + lda * Qi], floor_abs);
          }
          if (!__syncthreads_or(pend)) quiet = M;
        }
        if (quiet >= M) {
          converged = true;
          break;  // uniform: the counts come from block barriers
        }
        continue;
      }
      quiet = 0;
      // A <- J^T A J per 2 x 2 block (pair Pi rows, pair Qi columns, Pi <= Qi), mirrored
      for (int b = tid; b < nblk; b += kJ32NT) {
        const int pq = blk[b];
        const int Pi = pq & 0xffff, Qi = pq >> 16;
        const int wP = rpq[Pi], wQ = rpq[Qi];
        if (!((wP | wQ) >> 20)) continue;
        const int p1 = wP & 0x3ff, q1 = (wP >> 10) & 0x3ff, p2 = wQ & 0x3ff, q2 = (wQ >> 10) & 0x3ff;
        if (Pi == Qi) {
          const float app = A[p1 + lda * p1], aqq = A[q1 + lda * q1], apq = A[p1 + lda * q1];
          const float tt = rt[Pi];
          A[p1 + lda * p1] = app - tt * apq;
          A[q1 + lda * q1] = aqq + tt * apq;
          A[p1 + lda * q1] = 0.f;
          A[q1 + lda * p1] = 0.f;
          continue;
        }
        const float2 csP = rcs[Pi], csQ = rcs[Qi];
        const float cP = csP.x, sP = csP.y, cQ = csQ.x, sQ = csQ.y;
        const bool vp1 = p1 < n, vq1 = q1 < n, vp2 = p2 < n, vq2 = q2 < n;
        const float a = (vp1 && vp2) ? A[p1 + lda * p2] : 0.f;
        const float bb = (vp1 && vq2) ? A[p1 + lda * q2] : 0.f;
        const float c = (vq1 && vp2) ? A[q1 + lda * p2] : 0.f;
        const float d = (vq1 && vq2) ? A[q1 + lda * q2] : 0.f;
        const float y00 = a * cQ - bb * sQ, y01 = a * sQ + bb * cQ;
        const float y10 = c * cQ - d * sQ, y11 = c * sQ + d * cQ;
        const float x00 = cP * y00 - sP * y10, x01 = cP * y01 - sP * y11;
        const float x10 = sP * y00 + cP * y10, x11 = sP * y01 + cP * y11;
        if (vp1 && vp2) { A[p1 + lda * p2] = x00; A[p2 + lda * p1] = x00; }
        if (vp1 && vq2) { A[p1 + lda * q2] = x01; A[q2 + lda * p1] = x01; }
        if (vq1 && vp2) { A[q1 + lda * p2] = x10; A[p2 + lda * q1] = x10; }
        if (vq1 && vq2) { A[q1 + lda * q2] = x11; A[q2 + lda * q1] = x11; }
      }
      // V <- V J: one warp per rotated pair, lanes over the rows
      for (int pi = warp; pi < P; pi += NW) {
        const int w = rpq[pi];
        if (!(w >> 20)) continue;
        const int p = w & 0x3ff, q = (w >> 10) & 0x3ff;
        const float2 cs = rcs[pi];
        float* vp = V + lda * p;
        float* vq = V + lda * q;
        for (int row = lane; row < n; row += 32) {
          const float x = vp[row], y = vq[row];
          vp[row] = cs.x * x - cs.y * y;
          vq[row] = cs.y * x + cs.x * y;
        }
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < n * n; e += kJ32NT) {
    const int i = e % n, j = e / n;
    s.F32b[i + n * j] = V[i + lda * j];
  }
  if (tid == 0) s.eig_sweeps32 += sweep;
}

int jacobi32_smem_bytes(int n) {
  const int N = n + (n & 1), P = N / 2;
  return 2 * (N + 1) * N * 4 + P * (8 + 4 + 4) + (P * (P + 1) / 2) * 4 + 16;
}

void launch_eig_mixed(Search* S, TileMap tm32, int s0, int s1, int max_n, cudaStream_t st) {
  if (tm32.total <= 0 || s1 <= s0) return;
  const int g = tm32.total;
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_CB32);
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_BTT32);
  const int mn = max_n < kE32Max ? max_n : kE32Max;
  const int bytes = jacobi32_smem_bytes(mn);
  cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  k_jacobi32<<<s1 - s0, kJ32NT, bytes, st>>>(S, s0);
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_BV);    // ET = W = B V32
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_WTW);   // EA = (3I - W^T W)/2
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_WM);    // B = W EA
  k_eig_copy_b<<<g, 256, 0, st>>>(S, tm32);          // ET = B
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_WTW);   // second Newton-Schulz step
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_WM);
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_CW);    // ET = C B
  k_eig_stage<<<g, 256, 0, st>>>(S, tm32, OP_WTT);   // EA = B^T C B
}

}  // namespace cmaes_gb300
