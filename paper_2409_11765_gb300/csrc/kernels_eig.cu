// kernels_eig.cu -- lazy FP64 eigendecomposition C = B D^2 B^T (§2.1).
//
// The paper calls LAPACK's dsyev on the main process (§3.1). Here the
// decomposition is a warm-started parallel cyclic Jacobi method in FP64:
//   1. A = B^T C B with the previous eigenbasis B. Between two decompositions
//      C moves by O(c1 + c_mu), so A is nearly diagonal and few sweeps remain.
//   2. Round-robin (tournament) ordering: each step rotates N/2 disjoint
//      pairs (p, q) at once, chosen so that every pair meets once per sweep.
//      The rotation zeroing a_pq uses theta = (a_qq - a_pp) / (2 a_pq),
//      t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(1 + t^2),
//      s = t c (Golub & Van Loan, §8.5), and is skipped when
//      |a_pq| <= tol sqrt(|a_pp a_qq|) (a relative threshold); both are
//      evaluated by jacobi_rotation / jacobi_rotates (device_common.cuh),
//      which keep FP64 divides and square roots off the critical path.
//   3. A <- J^T A J is applied per 2 x 2 block (pair P rows, pair Q columns);
//      only blocks with P <= Q are computed and mirrored, so A stays
//      symmetric. B <- B J accumulates the rotations into the eigenbasis.
//   4. Sweeps repeat until one applies no rotation; then D^2 = diag(A), a PD
//      guard lifts eigenvalues below max * 1e-16, and BD = B diag(D).
//   5. The paper only asks for "a matrix containing orthonormal eigenvectors";
//      the representative is fixed here so that any two solvers agree: columns
//      in ascending eigenvalue order (ties by index) and each column's entry of
//      largest magnitude (first on ties) positive.
// Small n keeps A and B in shared memory (one CTA per search); larger n runs
// the same steps on the global-memory copies. For 32 < n <= kEigBigMaxN the
// warm start and most of the work belong to the refined route
// (kernels_eig_mixed.cu, kernels_eig_big.cu), and the global-memory variant
// (n > kJacobiClusterN) is its cleanup: it starts from A = X^T C X, nearly
// diagonal, and drives each step by the list of the pairs that rotate.
#include <cmath>
#include "device_common.cuh"

namespace cmaes_gb300 {

constexpr int kJacobiNT = 512;
constexpr double kJacobiTol = 1e-14;
constexpr int kJacobiMaxSweeps = 40;
constexpr double kPdFloor = 1e-16;

int jacobi_smem_bytes(int n, bool smem_mats) {
  const int N = n + (n & 1), P = N / 2;
  const int mats = smem_mats ? 2 * (N + 1) * N * 8 : 0;
  return mats + P * (3 * 8 + 4 * 4) + N * (2 * 8 + 4) + 16;
}

int jacobi_smem_max_n() {
  int best = 0;
  for (int n = 2; n <= 256; n += 2)
    if (jacobi_smem_bytes(n, true) <= 227 * 1024) best = n;
  return best;
}

// Searches whose warm start is prepared by the refined route
// (kernels_eig_mixed.cu) skip the FP64 B^T C B below.
// searches whose decomposition another route computes (the refined
// Jacobi route or the tridiagonal route) skip the plain warm start
__device__ __forceinline__ bool mixed_route(const Search& s) { return eig_refined_route(s) || s.trd; }

// ET = C B (square tiles; only searches whose decomposition is due).
__global__ void __launch_bounds__(256) k_eig_gemm_CB(Search* S, TileMap tm) {
  __shared__ GemmSmem sm;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !s.eig_due || mixed_route(s)) return;
  const int n = s.n, ldn = s.ldn, T = ceil_div(n, kGBM);
  const double* C = s.C;
  const double* B = s.B;
  double* ET = s.ET;
  gemm_tile_f64<true, true>(
      n, n, n, (t % T) * kGBM, (t / T) * kGBN,
      [=] __device__(int i, int k) { return C[i + static_cast<long long>(ldn) * k]; },
      [=] __device__(int k, int j) { return B[k + static_cast<long long>(ldn) * j]; },
      [=] __device__(int i, int j, double acc) { ET[i + static_cast<long long>(ldn) * j] = acc; }, sm);
}

// EA = B^T ET = B^T C B.
__global__ void __launch_bounds__(256) k_eig_gemm_BtT(Search* S, TileMap tm) {
  __shared__ GemmSmem sm;
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !s.eig_due || mixed_route(s)) return;
  const int n = s.n, ldn = s.ldn, T = ceil_div(n, kGBM);
  const double* B = s.B;
  const double* ET = s.ET;
  double* EA = s.EA;
  gemm_tile_f64<false, true>(
      n, n, n, (t % T) * kGBM, (t / T) * kGBN,
      [=] __device__(int i, int k) { return B[k + static_cast<long long>(ldn) * i]; },
      [=] __device__(int k, int j) { return ET[k + static_cast<long long>(ldn) * j]; },
      [=] __device__(int i, int j, double acc) { EA[i + static_cast<long long>(ldn) * j] = acc; }, sm);
}

void launch_eig_gemm_CB(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_eig_gemm_CB<<<tm.total, 256, 0, st>>>(S, tm);
}
void launch_eig_gemm_BtT(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_eig_gemm_BtT<<<tm.total, 256, 0, st>>>(S, tm);
}

// Pair i of round-robin step r over N players (player N-1 fixed).
__device__ __forceinline__ void rr_pair(int r, int i, int N, int& p, int& q) {
  const int M = N - 1;
  if (i == 0) {
    p = r;
    q = M;
  } else {
    p = (r + i) % M;
    q = (r - i + M) % M;
  }
}

template <bool SMEM>
__global__ void __launch_bounds__(kJacobiNT) k_jacobi(Search* S, int s0, int lo_n, int hi_n) {
  extern __shared__ double dsm[];
  __shared__ double shr[32];
  __shared__ long long sh_rot;
  __shared__ int sh_m;  // rotating pairs of the current step
  Search& s = S[s0 + blockIdx.x];
  if (s.done || !s.eig_due || s.trd) return;
  const int n = s.n, ldn = s.ldn;
  if (n <= lo_n || n > hi_n) return;
  const int N = n + (n & 1), P = N / 2;
  const int tid = threadIdx.x;
  double *A, *V;
  long long lda;
  double* rc;
  if (SMEM) {
    lda = N + 1;
    A = dsm;
    V = dsm + lda * N;
    rc = V + lda * N;
  } else {
    lda = ldn;
    A = s.EA;
    V = s.ET;  // free once EA = B^T (C B) is formed; B is rewritten at the end
    rc = dsm;
  }
  double* rsn = rc + P;
  double* rtn = rsn + P;
  double* ev = rtn + P;
  double* sg = ev + N;
  int* rp = reinterpret_cast<int*>(sg + N);
  int* rq = rp + P;
  int* ra = rq + P;
  int* rk = ra + P;
  int* al = rk + N;  // the rotating pairs of a step, in no particular order

  // symmetrised A = (EA + EA^T) / 2; V = B
  if (SMEM) {
    for (int e = tid; e < N * N; e += kJacobiNT) {
      const int i = e % N, j = e / N;
      double a = 0.0, v = 0.0;
      if (i < n && j < n) {
        a = 0.5 * (s.EA[i + static_cast<long long>(ldn) * j] + s.EA[j + static_cast<long long>(ldn) * i]);
        v = s.B[i + static_cast<long long>(ldn) * j];
      }
      A[i + lda * j] = a;
      V[i + lda * j] = v;
    }
  } else {
    for (long long e = tid; e < static_cast<long long>(n) * n; e += kJacobiNT) {
      const int i = static_cast<int>(e % n), j = static_cast<int>(e / n);
      if (i < j) {
        const double a = 0.5 * (A[i + lda * j] + A[j + lda * i]);
        A[i + lda * j] = a;
        A[j + lda * i] = a;
      }
      V[i + lda * j] = s.B[i + static_cast<long long>(ldn) * j];
    }
  }
  if (tid == 0) {
    sh_rot = 0;
    sh_m = 0;
  }
  __syncthreads();
  // The plain relative test on every handle, also as the cleanup of the
  // refined route (n > kJacobiClusterN here): at these sizes the FP32 stage
  // leaves pairs of close eigenvalues whose remains, if stopped at a rounding
  // floor of n eps64 max|a_ii|, add up to more than the 1e-12 reconstruction
  // error of the contract.
  const double floor_abs = 0.0;

  int sweeps = 0;
  // every pair meets once in any N - 1 consecutive steps, so N - 1 steps in a
  // row without a rotation mean convergence (same result as a quiet sweep)
  int quiet = 0;
  bool converged = false;
  for (; sweeps < kJacobiMaxSweeps && !converged; ++sweeps) {
    for (int r = 0; r < N - 1; ++r) {
      // rotations of this step
      int act_any = 0;
      for (int i = tid; i < P; i += kJacobiNT) {
        int p, q;
        rr_pair(r, i, N, p, q);
        double c = 1.0, sn = 0.0, tn = 0.0;
        int act = 0;
        if (p < n && q < n) {
          const double app = A[p + lda * p], aqq = A[q + lda * q], apq = A[p + lda * q];
          if (jacobi_rotates(app, aqq, apq, kJacobiTol * kJacobiTol, floor_abs)) {
            jacobi_rotation(app, aqq, apq, tn, c, sn);
            act = 1;
          }
        }
        rc[i] = c;
        rsn[i] = sn;
        rtn[i] = tn;
        rp[i] = p;
        rq[i] = q;
        ra[i] = act;
        if (act) {
          act_any = 1;
          atomicAdd(reinterpret_cast<unsigned long long*>(&sh_rot), 1ull);
          al[atomicAdd(&sh_m, 1)] = i;
        }
      }
      if (__syncthreads_count(act_any) == 0) {
        // a quiet step: if no off-diagonal entry passes the test any more, the
        // rest of the quiet window would change nothing
        ++quiet;
        // (on global memory a check reads all of A: at the 64th quiet step and
        // every 256th after it, so that isolated rotating steps, as in a
        // cleanup, do not each cost a pass over the matrix)
        if (SMEM ? (quiet == 1 || quiet % 16 == 0) : (quiet == 64 || quiet % 256 == 0)) {
          int pend = 0;
          for (int j = tid >> 5; j < n && !pend; j += kJacobiNT / 32) {
            const double ajj = A[j + lda * j];
            for (int i = tid & 31; i < j; i += 32)
              pend |= jacobi_rotates(A[i + lda * i], ajj, A[i + lda * j], kJacobiTol * kJacobiTol, floor_abs);
          }
          if (!__syncthreads_or(pend)) quiet = N - 1;
        }
        if (quiet >= N - 1) {
          converged = true;
          break;  // uniform over the block: the counts come from block barriers
        }
        continue;
      }
      quiet = 0;
      const int m = sh_m;
      if (!SMEM && 6LL * m * n < static_cast<long long>(P) * P) {
        // Few rotations (as in a cleanup after the refinement): the m pairs'
        // columns of A, then their rows, then their exact 2 x 2 blocks, then
        // V's columns, O(m n) instead of a pass over every block. Pairs are
        // disjoint, so each entry gets at most one column and one row
        // rotation, in that order, whatever the order of the list.
        double* pre = ev;  // free until the eigenvalues: a_pp, a_qq, a_pq before the step
        for (int k = tid; k < m; k += kJacobiNT) {
          const int i = al[k], p = rp[i], q = rq[i];
          pre[3 * k] = A[p + lda * p];
          pre[3 * k + 1] = A[q + lda * q];
          pre[3 * k + 2] = A[p + lda * q];
        }
        __syncthreads();
        for (long long e = tid; e < static_cast<long long>(m) * n; e += kJacobiNT) {  // A <- A J
          const int k = static_cast<int>(e / n), r = static_cast<int>(e % n);
          const int i = al[k], p = rp[i], q = rq[i];
          const double c = rc[i], sn = rsn[i], x = A[r + lda * p], y = A[r + lda * q];
          A[r + lda * p] = c * x - sn * y;
          A[r + lda * q] = sn * x + c * y;
        }
        __syncthreads();
        for (long long e = tid; e < static_cast<long long>(m) * n; e += kJacobiNT) {  // A <- J^T A
          const int k = static_cast<int>(e / n), col = static_cast<int>(e % n);
          const int i = al[k], p = rp[i], q = rq[i];
          const double c = rc[i], sn = rsn[i], x = A[p + lda * col], y = A[q + lda * col];
          A[p + lda * col] = c * x - sn * y;
          A[q + lda * col] = sn * x + c * y;
        }
        __syncthreads();
        for (int k = tid; k < m; k += kJacobiNT) {  // the exact 2 x 2 diagonal blocks
          const int i = al[k], p = rp[i], q = rq[i];
          const double t = rtn[i], app = pre[3 * k], aqq = pre[3 * k + 1], apq = pre[3 * k + 2];
          A[p + lda * p] = app - t * apq;
          A[q + lda * q] = aqq + t * apq;
          A[p + lda * q] = 0.0;
          A[q + lda * p] = 0.0;
        }
        for (long long e = tid; e < static_cast<long long>(m) * n; e += kJacobiNT) {  // V <- V J
          const int k = static_cast<int>(e / n), row = static_cast<int>(e % n);
          const int i = al[k], p = rp[i], q = rq[i];
          const double c = rc[i], sn = rsn[i], vp = V[row + lda * p], vq = V[row + lda * q];
          V[row + lda * p] = c * vp - sn * vq;
          V[row + lda * q] = sn * vp + c * vq;
        }
        if (tid == 0) sh_m = 0;
        __syncthreads();
        continue;
      }
      // A <- J^T A J per 2x2 block (P <= Q), mirrored
      const int nblk = P * (P + 1) / 2;
      // row-major enumeration of the upper triangle of the P x P block grid:
      // b = Qi (Qi + 1) / 2 + Pi, Pi <= Qi
      auto block_of = [](int b, int& Pi, int& Qi) {
        int bp = static_cast<int>((sqrtf(static_cast<float>(8 * b + 1)) - 1.0f) * 0.5f);
        while ((bp + 1) * (bp + 2) / 2 <= b) ++bp;
        while (bp * (bp + 1) / 2 > b) --bp;
        Pi = b - bp * (bp + 1) / 2;
        Qi = bp;
      };
      if (SMEM) {
        for (int b = tid; b < nblk; b += kJacobiNT) {
          int Pi, Qi;
          block_of(b, Pi, Qi);
          const int aP = ra[Pi], aQ = ra[Qi];
          if (!aP && !aQ) continue;
          const int p1 = rp[Pi], q1 = rq[Pi], p2 = rp[Qi], q2 = rq[Qi];
          if (Pi == Qi) {
            const double app = A[p1 + lda * p1], aqq = A[q1 + lda * q1], apq = A[p1 + lda * q1];
            const double t = rtn[Pi];
            A[p1 + lda * p1] = app - t * apq;
            A[q1 + lda * q1] = aqq + t * apq;
            A[p1 + lda * q1] = 0.0;
            A[q1 + lda * p1] = 0.0;
            continue;
          }
          const double cP = rc[Pi], sP = rsn[Pi], cQ = rc[Qi], sQ = rsn[Qi];
          const bool vp1 = p1 < n, vq1 = q1 < n, vp2 = p2 < n, vq2 = q2 < n;
          const double a = (vp1 && vp2) ? A[p1 + lda * p2] : 0.0;
          const double bb = (vp1 && vq2) ? A[p1 + lda * q2] : 0.0;
          const double c = (vq1 && vp2) ? A[q1 + lda * p2] : 0.0;
          const double d = (vq1 && vq2) ? A[q1 + lda * q2] : 0.0;
          const double y00 = a * cQ - bb * sQ, y01 = a * sQ + bb * cQ;
          const double y10 = c * cQ - d * sQ, y11 = c * sQ + d * cQ;
          const double x00 = cP * y00 - sP * y10, x01 = cP * y01 - sP * y11;
          const double x10 = sP * y00 + cP * y10, x11 = sP * y01 + cP * y11;
          if (vp1 && vp2) { A[p1 + lda * p2] = x00; A[p2 + lda * p1] = x00; }
          if (vp1 && vq2) { A[p1 + lda * q2] = x01; A[q2 + lda * p1] = x01; }
          if (vq1 && vp2) { A[q1 + lda * p2] = x10; A[p2 + lda * q1] = x10; }
          if (vq1 && vq2) { A[q1 + lda * q2] = x11; A[q2 + lda * q1] = x11; }
        }
        // V <- V J for the active pairs
        for (long long e = tid; e < static_cast<long long>(P) * n; e += kJacobiNT) {
          const int pi = static_cast<int>(e / n), row = static_cast<int>(e % n);
          if (!ra[pi]) continue;
          const int p = rp[pi], q = rq[pi];
          const double c = rc[pi], sn = rsn[pi];
          const double vp = V[row + lda * p], vq = V[row + lda * q];
          V[row + lda * p] = c * vp - sn * vq;
          V[row + lda * q] = sn * vp + c * vq;
        }
      } else {
        // On global memory the step is driven by the list of its m rotating
        // pairs: warp w takes pairs al[w], al[w + NW], ... and its lanes the
        // partner pairs, so only the blocks with a rotating pair are visited
        // (each once: a block of two rotating pairs belongs to the lower
        // one), and V's rows follow the same pairs. No integer division and
        // no pass over idle blocks, whatever m is.
        constexpr int NW = kJacobiNT / 32;
        const int lane = tid & 31, warp = tid >> 5;
        for (int k = warp; k < m; k += NW) {
          const int a = al[k];
          for (int j = lane; j < P; j += 32) {
            if (ra[j] && j < a) continue;  // that block is pair j's
            const int Pi = j < a ? j : a, Qi = j < a ? a : j;
            const int p1 = rp[Pi], q1 = rq[Pi], p2 = rp[Qi], q2 = rq[Qi];
            if (Pi == Qi) {  // the pair's own 2 x 2 block, set exactly
              const double app = A[p1 + lda * p1], aqq = A[q1 + lda * q1], apq = A[p1 + lda * q1];
              const double t = rtn[Pi];
              A[p1 + lda * p1] = app - t * apq;
              A[q1 + lda * q1] = aqq + t * apq;
              A[p1 + lda * q1] = 0.0;
              A[q1 + lda * p1] = 0.0;
              continue;
            }
            const double cP = rc[Pi], sP = rsn[Pi], cQ = rc[Qi], sQ = rsn[Qi];
            const bool vp1 = p1 < n, vq1 = q1 < n, vp2 = p2 < n, vq2 = q2 < n;
            const double x0 = (vp1 && vp2) ? A[p1 + lda * p2] : 0.0;
            const double x1 = (vp1 && vq2) ? A[p1 + lda * q2] : 0.0;
            const double x2 = (vq1 && vp2) ? A[q1 + lda * p2] : 0.0;
            const double x3 = (vq1 && vq2) ? A[q1 + lda * q2] : 0.0;
            const double y00 = x0 * cQ - x1 * sQ, y01 = x0 * sQ + x1 * cQ;
            const double y10 = x2 * cQ - x3 * sQ, y11 = x2 * sQ + x3 * cQ;
            const double x00 = cP * y00 - sP * y10, x01 = cP * y01 - sP * y11;
            const double x10 = sP * y00 + cP * y10, x11 = sP * y01 + cP * y11;
            if (vp1 && vp2) { A[p1 + lda * p2] = x00; A[p2 + lda * p1] = x00; }
            if (vp1 && vq2) { A[p1 + lda * q2] = x01; A[q2 + lda * p1] = x01; }
            if (vq1 && vp2) { A[q1 + lda * p2] = x10; A[p2 + lda * q1] = x10; }
            if (vq1 && vq2) { A[q1 + lda * q2] = x11; A[q2 + lda * q1] = x11; }
          }
          // V <- V J for pair a: its two columns, lanes over the rows
          const int p = rp[a], q = rq[a];
          const double c = rc[a], sn = rsn[a];
          for (int row = lane; row < n; row += 32) {
            const double vp = V[row + lda * p], vq = V[row + lda * q];
            V[row + lda * p] = c * vp - sn * vq;
            V[row + lda * q] = sn * vp + c * vq;
          }
        }
      }
      if (tid == 0) sh_m = 0;
      __syncthreads();
    }
  }

  // eigenvalues with the PD guard
  double lo = INFINITY, hi = -INFINITY;
  for (int i = tid; i < n; i += kJacobiNT) {
    const double e = A[i + lda * i];
    lo = fmin(lo, e);
    hi = fmax(hi, e);
  }
  hi = block_max<kJacobiNT>(hi, shr);
  lo = -block_max<kJacobiNT>(-lo, shr);
  const double add = (lo < hi * kPdFloor) ? hi * kPdFloor - lo : 0.0;
  for (int i = tid; i < n; i += kJacobiNT) {
    ev[i] = A[i + lda * i] + add;
    if (add != 0.0) s.C[i + static_cast<long long>(ldn) * i] += add;
  }
  __syncthreads();
  // canonical representative: rank by ascending eigenvalue (ties by index) ...
  for (int i = tid; i < n; i += kJacobiNT) {
    const double e = ev[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (ev[j] < e) || (ev[j] == e && j < i);
    rk[i] = r;
  }
  // ... and the sign that makes the largest-magnitude entry positive
  const int lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < n; j += kJacobiNT / 32) {
    double best = -1.0, val = 0.0;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      const double v = V[i + lda * j], a = fabs(v);
      if (a > best) { best = a; val = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const double ov = __shfl_xor_sync(0xffffffffu, val, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; val = ov; bi = oi; }
    }
    if (lane == 0) sg[j] = (val < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += kJacobiNT) s.D[rk[i]] = sqrt(ev[i]);
  for (long long e = tid; e < static_cast<long long>(n) * n; e += kJacobiNT) {
    const int i = static_cast<int>(e % n), j = static_cast<int>(e / n);
    s.B[i + static_cast<long long>(ldn) * rk[j]] = sg[j] * V[i + lda * j];
  }
  if (tid == 0) {
    const int done_sweeps = sweeps;
    s.eig_sweeps = done_sweeps;
    s.eig_count += 1;
    s.eig_sweeps_total += done_sweeps;
    s.eig_rotations += sh_rot;
  }
}

// Each launch covers the whole search range and processes the searches with
// lo_n < n <= hi_n (A and B in shared memory needs hi_n <= jacobi_smem_max_n()).
void launch_jacobi_variant(Search* S, int s0, int s1, bool smem, int lo_n, int hi_n, int max_n,
                           cudaStream_t st) {
  if (s1 <= s0 || max_n <= lo_n) return;
  const int bytes = jacobi_smem_bytes(max_n, smem);
  if (smem) {
    cudaFuncSetAttribute(k_jacobi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    k_jacobi<true><<<s1 - s0, kJacobiNT, bytes, st>>>(S, s0, lo_n, hi_n);
  } else {
    cudaFuncSetAttribute(k_jacobi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    k_jacobi<false><<<s1 - s0, kJacobiNT, bytes, st>>>(S, s0, lo_n, hi_n);
  }
}

// BD = B diag(D); force = 1 applies to every search (after set_state).
__global__ void __launch_bounds__(256) k_set_bd(Search* S, TileMap tm, int force) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (s.done || !(force || s.eig_due)) return;
  const int n = s.n, ldn = s.ldn, T = ceil_div(n, 64);
  const int i0 = (t % T) * 64, j0 = (t / T) * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int i = i0 + (e & 63), j = j0 + (e >> 6);
    if (i < n && j < n) {
      const long long x = i + static_cast<long long>(ldn) * j;
      s.BD[x] = s.B[x] * s.D[j];
    }
  }
}

void launch_set_bd(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_set_bd<<<tm.total, 256, 0, st>>>(S, tm, 0);
}
void launch_set_bd_force(Search* S, TileMap tm, cudaStream_t st) {
  if (tm.total > 0) k_set_bd<<<tm.total, 256, 0, st>>>(S, tm, 1);
}

}  // namespace cmaes_gb300
