// kernels_eig_trd.cu -- the tridiagonal route of the eigendecomposition
// C = B D^2 B^T (32 < n <= kEigBigMaxN; the default route).
//
// The paper computes B and D with LAPACK's dsyev (§3.1), i.e. Householder
// reduction to tridiagonal form followed by a tridiagonal eigensolver. On
// GB300 FP64 issues at 1/64 of the FP32 rate, so the route is built for few
// FP64 flops and few sequential steps, all in FP64 (no refinement needed):
//   1. Householder tridiagonalisation T = Q^T C Q (unblocked, lower part;
//      Golub & Van Loan §8.3.1), by a group of CTAs per search in one
//      cooperative launch: per step every CTA of the group forms the reflector
//      of column k itself (the same fixed-order arithmetic everywhere), then
//      each CTA applies the pending rank-2 update A <- A - v w^T - w v^T of the
//      previous step to the columns it owns while it accumulates the symmetric
//      product p = tau A v for the new v: one pass over the trailing matrix and
//      one group barrier per step.
//   2. Splitting: off-diagonal entries below 4 sqrt(n) eps64 ||T|| are set to
//      zero, which cuts T into independent blocks (this is where the repeated
//      eigenvalues of a low-rank update of a multiple of I separate).
//   3. Eigenvalues of each block by bisection on Sturm counts (one thread per
//      eigenvalue), to an absolute accuracy of 4 eps64 ||T||.
//   4. Eigenvectors of each block by inverse iteration (Gaussian elimination
//      with partial pivoting on T - lambda I, three solves from a
//      pseudo-random start); vectors of one block whose eigenvalues lie within
//      1e-13 ||T|| of each other (where inverse iteration may return nearly
//      parallel vectors) are orthogonalised by Gram-Schmidt (twice; classical
//      on a whole CTA for long chunks, modified on one warp for short ones),
//      in chunks of at most 64 consecutive vectors: a longer chain is a
//      repeated eigenvalue spread by rounding, whose vectors come from
//      independent pseudo-random starts and overlap little across chunks.
//   5. Newton-Schulz steps V <- V + V (I - V^T V) / 2 restore orthogonality
//      to rounding: inverse iteration leaves pairs with small absolute gaps
//      (the small eigenvalues of an ill-conditioned C, the spread-out copies
//      of a repeated eigenvalue) off by about eps64 ||T|| / gap, at most
//      ~1e-3 outside the Gram-Schmidt clusters. V^T V is formed in FP64, the
//      correction (of the size of that defect) in FP32; up to three steps,
//      each after the first only when the previous one started from a defect
//      above 5e-9.
//   6. Back-transformation B = Q V with the stored reflectors, then the
//      canonical form shared with the Jacobi route: columns in ascending
//      eigenvalue order, each column's entry of largest magnitude positive,
//      the PD guard on the eigenvalues.
// Every reduction has a fixed order, so a search gives the same bits alone
// and inside any batch.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include "device_common.cuh"
#include "ozaki.cuh"
#include "trd_common.cuh"

namespace cmaes_gb300 {

__device__ __forceinline__ double warp_sum_xor(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of the G CTAs of one search. The launch is cooperative, so every
// CTA of the group is resident; the wait is still bounded: after ~1 s the
// device status word records a time-out and the CTA leaves the reduction.
__device__ bool trd_group_sync(unsigned* ctr, unsigned target, int* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const long long t0 = clock64();
    int ok = 1;
    while (ld_acquire_u32(ctr) < target) {
      if (clock64() - t0 > kTrdWaitCycles) {
        atomicOr(err, kDevErrTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *sh_ok = ok;
  }
  __syncthreads();
  return *sh_ok != 0;
}

// --------------------------------------------------------------------------
// 1. Householder tridiagonalisation in panels of kPnb columns (the blocked
// form of LAPACK's dsytrd / dlatrd). Within panel [k0, k1) the matrix A (EA)
// is only read: the current matrix is A - V W^T - W V^T with V the panel's
// reflectors so far (columns k0.. of EX) and W (columns 0.. of EG) built step
// by step; after the panel the trailing part of A takes that rank-2 kPnb
// update as FP64-accurate products on the tensor cores (k_trd_s2k_*).
// CTA blockIdx.x works for search grp[b].x as member r = grp[b].y of a group
// of G = grp[b].z CTAs: it owns the 32-row chunks c with c mod G = r (the
// column products are dealt at run time). Step k (panel column j = k - k0) in
// two phases:
//   A. with u_W = W^T v, u_V = V^T v (the previous step's v, from the previous
//      phase B) and q = A v on the own rows, the previous step's
//      p = tau (q - V u_W - W u_V) and w = p - (tau / 2)(p . v) v, where
//      p . v = tau (q . v - 2 u_W . u_V); then, in the same pass over the own
//      rows, column k of the current matrix, c = A(:, k) - V W(k, :)^T -
//      W V(k, :)^T (to cbuf), and the partial sum of |c(k+2:)|^2;
//                                                               group barrier
//   B. (every CTA) the reflector of c and its vector v; then the products
//      q(j') = A(:, j')^T v (to qbuf, and q(j') v(j') to qv) and
//      u = [W V]^T v over rows k+1.., column pairs dealt to the group's warps
//      from a per-step counter; q . v is summed in phase A of the next step
//      over all rows by all warps, in a fixed order;
//                                                               group barrier
// The group (its size may differ from panel to panel) counts its barriers
// from the start of the panel: barrier m waits for G m arrivals; in panel 0
// the one after the symmetrisation is m = 1 and step k's are 2k + 2 and
// 2k + 3, in the others step k's are 2(k - k0) + 1 and 2(k - k0) + 2.
// Dynamic shared memory: v (n doubles).
// --------------------------------------------------------------------------
constexpr int kUbuf = 2 * kPnb;  // u_W then u_V at the start of Search::EH, then the partial sums

__global__ void __launch_bounds__(kTrdNT, 4) k_trd_panel(Search* S, const int4* grp, int q) {
  extern __shared__ double vsm[];
  __shared__ double sVk[kPnb], sWk[kPnb], su[2 * kPnb];
  __shared__ double red[kTrdNT / 32 + 8];
  __shared__ int sh_ok;
  const int4 g = grp[blockIdx.x];
  Search& s = S[g.x];
  if (!trd_due(s)) return;
  const int n = s.n, k0 = kPnb * q;
  if (k0 >= n) return;
  const int k1 = min(k0 + kPnb, n);
  const long long L = s.ldn;
  const int r = g.y, G = g.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kTrdNT / 32;
  double* A = s.EA;
  double* Hv = s.EX;
  double* Wp = s.EG;
  double* d = tv(s, TV_D);
  double* e = tv(s, TV_E);
  double* tau = tv(s, TV_TAU);
  double* cbuf = tv(s, TV_P0);
  double* qbuf = tv(s, TV_P1);
  double* qv = tv(s, TV_SD);          // q(j) v(j) per column
  double* ubuf = s.EH;                // u_W (kPnb), u_V (kPnb)
  double* part = s.EH + kUbuf;        // per-CTA partial |c|^2, kPartStride apart
  unsigned* bar = s.trd_bar;
  auto barrier = [&](unsigned m) -> bool {
    if (G > 1) return trd_group_sync(bar, static_cast<unsigned>(G) * m, s.err, &sh_ok);
    __syncthreads();
    return true;
  };
  if (q == 0) {  // A = (C + C^T) / 2, owned columns
    const double* C = s.C;
    for (int jc = r; jc < n; jc += G)
      for (int i = tid; i < n; i += kTrdNT) A[i + L * jc] = 0.5 * (C[i + L * jc] + C[jc + L * i]);
    if (!barrier(1u)) return;
  }
  // the first own 32-row chunk at or after row `row`
  auto first_chunk = [&](int row) {
    const int c0 = row >> 5;
    return c0 + ((r - c0 % G) % G + G) % G;
  };
  const unsigned mbase = q == 0 ? 1u : 0u;
  double tprev = 0.0;
  // Phase A of step k (j = k - k0); with last, only the previous step's w on
  // the own rows i >= k (the end of the panel). Returns the partial |c|^2.
  auto phase_a = [&](int k, int j, bool last) -> double {
    const int jp = j - 1;  // columns of W and V before the previous step
    if (j > 0) {
      for (int l = tid; l < jp; l += kTrdNT) {
        su[l] = __ldcg(&ubuf[l]);
        su[kPnb + l] = __ldcg(&ubuf[kPnb + l]);
        sVk[l] = __ldcg(&Hv[k + L * (k0 + l)]);
        sWk[l] = __ldcg(&Wp[k + L * l]);
      }
      {  // q . v: warp w sums rows k + 32 w + lane + 256 m (two chains), in fixed order
        double s0 = 0.0, s1 = 0.0;
        int c = k + 32 * warp + lane;
        for (; c + kTrdNT < n; c += 2 * kTrdNT) {
          s0 += __ldcg(&qv[c]);
          s1 += __ldcg(&qv[c + kTrdNT]);
        }
        if (c < n) s0 += __ldcg(&qv[c]);
        const double sw = warp_sum_xor(s0 + s1);
        if (lane == 0) red[warp] = sw;
      }
      __syncthreads();
      if (warp == 0) {  // u_W . u_V and the row-k correction, lanes in fixed order
        double uu = 0.0, ck = 0.0;
        for (int l = lane; l < jp; l += 32) {
          uu = fma(su[l], su[kPnb + l], uu);
          ck = fma(sVk[l], su[l], fma(sWk[l], su[kPnb + l], ck));
        }
        uu = warp_sum_xor(uu);
        ck = warp_sum_xor(ck);
        if (lane == 0) {
          double sq = 0.0;
          for (int w = 0; w < NW; ++w) sq += red[w];
          const double half = 0.5 * tprev * tprev * (sq - 2.0 * uu);  // (tau / 2) p . v
          const double pk = tprev * (__ldcg(&qbuf[k]) - ck);
          sVk[jp] = 1.0;                // v_{k-1}(k)
          sWk[jp] = fma(-half, 1.0, pk);  // w_{k-1}(k)
          red[NW] = half;
        }
      }
      __syncthreads();
    }
    const double half = j > 0 ? red[NW] : 0.0;
    double nrm = 0.0;
    for (int c = first_chunk(k) + G * warp; 32 * c < n; c += G * NW) {
      const int i = 32 * c + lane;
      if (i < k || i >= n) continue;
      // V u_W + W u_V (previous step), then the column correction: two
      // chains each (even and odd columns of every group of eight), summed last
      double pc0 = 0.0, pc1 = 0.0, cc0 = 0.0, cc1 = 0.0;
      int l = 0;
      for (; l + 8 <= jp; l += 8) {  // eight columns' loads in flight
        double hv[8], wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          hv[u] = __ldcg(&Hv[i + L * (k0 + l + u)]);
          wv[u] = __ldcg(&Wp[i + L * (l + u)]);
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          pc0 = fma(hv[u], su[l + u], fma(wv[u], su[kPnb + l + u], pc0));
          cc0 = fma(hv[u], sWk[l + u], fma(wv[u], sVk[l + u], cc0));
          pc1 = fma(hv[u + 1], su[l + u + 1], fma(wv[u + 1], su[kPnb + l + u + 1], pc1));
          cc1 = fma(hv[u + 1], sWk[l + u + 1], fma(wv[u + 1], sVk[l + u + 1], cc1));
        }
      }
      for (; l < jp; ++l) {
        const double hv = __ldcg(&Hv[i + L * (k0 + l)]), wv = __ldcg(&Wp[i + L * l]);
        pc0 = fma(hv, su[l], fma(wv, su[kPnb + l], pc0));
        cc0 = fma(hv, sWk[l], fma(wv, sVk[l], cc0));
      }
      const double pc = pc0 + pc1;
      double cc = cc0 + cc1;
      if (j > 0) {
        const double vi = vsm[i];  // v_{k-1}(i)
        const double wi = fma(-half, vi, tprev * (__ldcg(&qbuf[i]) - pc));
        Wp[i + L * jp] = wi;
        cc = fma(vi, sWk[jp], fma(wi, sVk[jp], cc));
      }
      if (!last && i > k) {
        const double ci = __ldcg(&A[i + L * k]) - cc;
        vsm[i] = ci;
        cbuf[i] = ci;
        if (i >= k + 2) nrm = fma(ci, ci, nrm);
      }
    }
    return nrm;
  };
  for (int k = k0; k < k1; ++k) {
    const int j = k - k0;
    // ---------------- A ----------------
    double nrm = phase_a(k, j, false);
    if (k == n - 1) {  // the last diagonal entry
      if (r == 0 && tid == 0) {
        double acc = __ldcg(&A[k + L * k]);
        for (int l = 0; l < j; ++l) acc = fma(-2.0 * sVk[l], sWk[l], acc);
        d[k] = acc;
      }
      return;
    }
    nrm = warp_sum_xor(nrm);
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int w = 0; w < NW; ++w) a += red[w];
      part[static_cast<long long>(r) * kPartStride] = a;
    }
    if (!barrier(mbase + 2u * j + 1u)) return;
    // ---------------- B ----------------
    if (warp == 0) {
      double a = 0.0;
      for (int c = lane; c < G; c += 32) a += __ldcg(&part[static_cast<long long>(c) * kPartStride]);
      a = warp_sum_xor(a);
      if (lane == 0) red[NW + 1] = a;
    }
    if (warp == 1) {  // the diagonal entry of column k: A(k, k) - 2 V(k, :) W(k, :)^T
      double acc = 0.0;
      for (int l = lane; l < j; l += 32) acc = fma(sVk[l], sWk[l], acc);
      acc = warp_sum_xor(acc);
      if (lane == 0) red[NW + 2] = fma(-2.0, acc, __ldcg(&A[k + L * k]));
    }
    if (tid == 64) red[NW + 5] = __ldcg(&cbuf[k + 1]);  // alpha
    __syncthreads();
    if (tid == 0) {
      const double xn2 = red[NW + 1];
      const double alpha = red[NW + 5];
      double t = 0.0, beta = alpha, scale = 0.0;
      if (xn2 > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
        t = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      red[NW] = t;
      red[NW + 3] = scale;
      if (r == 0) {
        d[k] = red[NW + 2];
        e[k] = beta;
        tau[k] = t;
      }
    }
    __syncthreads();
    const double t = red[NW], scale = red[NW + 3];
    for (int i = k + 1 + tid; i < n; i += kTrdNT) vsm[i] = (i == k + 1) ? 1.0 : __ldcg(&cbuf[i]) * scale;
    __syncthreads();
    for (int c = first_chunk(k + 1) + G * warp; 32 * c < n; c += G * NW) {
      const int i = 32 * c + lane;
      if (i > k && i < n) Hv[i + L * k] = vsm[i];
    }
    // columns j' >= k + 1 of A two at a time, then the 2j columns of [W V]
    // two at a time (u = [W V]^T v over rows k+1..), dealt at run time to the
    // group's warps from the step's work counter (the next pair is claimed
    // before the current one is worked)
    {
      unsigned* wctr = bar + 1 + j;
      const int units_a = (n - k) >> 1;  // pairs (k+1, k+2), (k+3, k+4), ...; the last may be single
      const int units = units_a + j;
      int u = 0;
      if (lane == 0) u = static_cast<int>(atomicAdd(wctr, 1u));
      u = __shfl_sync(0xffffffffu, u, 0);
      while (u < units) {
        int un = 0;
        if (lane == 0) un = static_cast<int>(atomicAdd(wctr, 1u));
        const bool is_a = u < units_a;
        int j1, j2;            // A: columns j1, j2; [W V]: entries j1, j2 of the 2j
        const double *A1, *A2;
        bool two = true;
        if (is_a) {
          j1 = k + 1 + 2 * u;
          j2 = j1 + 1;
          two = j2 < n;
          A1 = A + L * j1;
          A2 = A + L * (two ? j2 : j1);
        } else {
          j1 = 2 * (u - units_a);
          j2 = j1 + 1;
          A1 = j1 < j ? Wp + L * j1 : Hv + L * (k0 + j1 - j);
          A2 = j2 < j ? Wp + L * j2 : Hv + L * (k0 + j2 - j);
        }
        double q1 = 0.0, q2 = 0.0;
        int i = k + 1 + lane;
        constexpr int U = 8;  // rows per lane in flight, two columns
        for (; i + 32 * (U - 1) < n; i += 32 * U) {
          double a1[U], a2[U];
#pragma unroll
          for (int uu = 0; uu < U; ++uu) {
            a1[uu] = __ldcg(&A1[i + 32 * uu]);
            a2[uu] = two ? __ldcg(&A2[i + 32 * uu]) : 0.0;
          }
#pragma unroll
          for (int uu = 0; uu < U; ++uu) {
            const double vi = vsm[i + 32 * uu];
            q1 = fma(a1[uu], vi, q1);
            q2 = fma(a2[uu], vi, q2);
          }
        }
        for (; i < n; i += 32) {
          const double vi = vsm[i];
          q1 = fma(__ldcg(&A1[i]), vi, q1);
          if (two) q2 = fma(__ldcg(&A2[i]), vi, q2);
        }
        // both sums in one tree: the first level leaves column 1's pairs on
        // lanes 0-15 and column 2's on lanes 16-31 (five FP64 adds, not ten)
        const bool hi = (lane & 16) != 0;
        double qs = (hi ? q2 : q1) + __shfl_xor_sync(0xffffffffu, hi ? q1 : q2, 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
        const int jw = lane == 0 ? j1 : j2;
        if ((lane == 0 || (lane == 16 && two)) && is_a) {
          qbuf[jw] = qs;
          qv[jw] = qs * vsm[jw];
        } else if ((lane == 0 || lane == 16) && !is_a) {
          ubuf[jw < j ? jw : kPnb + jw - j] = qs;
        }
        u = __shfl_sync(0xffffffffu, un, 0);
      }
    }
    if (!barrier(mbase + 2u * j + 2u)) return;
    tprev = t;
  }
  // the panel's last w (its last step was a full one: k1 < n)
  phase_a(k1, k1 - k0, true);
}

// --------------------------------------------------------------------------
// 1'. The unblocked reduction, for handles whose searches leave the GPU
// partly idle (each group at its largest size): then a step's latency, not
// the FP64 work, sets the time, and this form has one group barrier per step
// (against two in the panel form). Golub & Van Loan §8.3.1: per step every
// CTA forms the reflector of column k itself (the same fixed-order
// arithmetic everywhere), then applies the pending rank-2 update
// A <- A - v w^T - w v^T of the previous step to the columns it owns while it
// accumulates p = tau A v for the new v: one pass over the trailing matrix.
// CTA blockIdx.x works for search grp[b].x as member grp[b].y of a group of
// grp[b].z CTAs; column j belongs to member j mod G, and within it to warp
// (j div G) mod 8. Dynamic shared memory: v and w of the previous step and v
// of the current one (3 n doubles).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrdNT) k_trd_sytrd(Search* S, const int4* grp) {
  extern __shared__ double tsm[];
  __shared__ double red[kTrdNT / 32 + 8];
  __shared__ int sh_ok;
  const int4 g = grp[blockIdx.x];
  Search& s = S[g.x];
  if (!trd_due(s)) return;
  const int n = s.n;
  const long long L = s.ldn;
  const int r = g.y, G = g.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kTrdNT / 32;
  double* W = s.EA;
  double* Hv = s.EX;
  const double* C = s.C;
  double* d = tv(s, TV_D);
  double* e = tv(s, TV_E);
  double* tau = tv(s, TV_TAU);
  double* pbuf = tv(s, TV_P0);  // two buffers: step k uses pbuf + (k & 1) L
  double* sdot = tv(s, TV_SD);  // per-CTA partial p.v, two buffers of L / 2
  unsigned* bar = s.trd_bar;
  double* vprev = tsm;
  double* wprev = tsm + n;
  double* vcur = tsm + 2 * n;
  // W = (C + C^T) / 2, owned columns only
  for (int j = r; j < n; j += G)
    for (int i = tid; i < n; i += kTrdNT) W[i + L * j] = 0.5 * (C[i + L * j] + C[j + L * i]);
  for (int i = tid; i < n; i += kTrdNT) {
    vprev[i] = 0.0;
    wprev[i] = 0.0;
  }
  unsigned nb = 0;
  if (G > 1) {
    if (!trd_group_sync(bar, G * ++nb, s.err, &sh_ok)) return;
  } else {
    __syncthreads();
  }
  for (int k = 0; k + 1 < n; ++k) {
    // column k with the pending update of step k - 1
    for (int i = k + tid; i < n; i += kTrdNT)
      vcur[i] = fma(-wprev[i], vprev[k], fma(-vprev[i], wprev[k], __ldcg(&W[i + L * k])));
    __syncthreads();
    // its reflector (warp 0, fixed-order sum)
    if (warp == 0) {
      double part = 0.0;
      for (int i = k + 2 + lane; i < n; i += 32) part = fma(vcur[i], vcur[i], part);
      const double xn2 = warp_sum_xor(part);
      if (lane == 0) {
        const double alpha = vcur[k + 1];
        double t = 0.0, beta = alpha, scale = 0.0;
        if (xn2 > 0.0) {
          beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
          t = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        red[NW] = t;
        red[NW + 1] = beta;
        red[NW + 2] = scale;
        red[NW + 3] = vcur[k];
      }
    }
    __syncthreads();
    const double t = red[NW], scale = red[NW + 2];
    for (int i = k + 2 + tid; i < n; i += kTrdNT) vcur[i] *= scale;
    if (tid == 0) vcur[k + 1] = 1.0;
    __syncthreads();
    if (r == 0) {
      for (int i = k + 1 + tid; i < n; i += kTrdNT) Hv[i + L * k] = vcur[i];
      if (tid == 0) {
        d[k] = red[NW + 3];
        e[k] = red[NW + 1];
        tau[k] = t;
      }
    }
    // owned columns j >= k + 1, two per warp at a time: pending update, then
    // p_j = tau (A v)_j, and this CTA's share of p . v
    double* pk = pbuf + (k & 1) * L;
    const int m0 = (k + 1 > r) ? (k + 1 - r + G - 1) / G : 0;
    double pv = 0.0;
    for (int m = m0 + warp;; m += 2 * NW) {
      const int j1 = r + G * m, j2 = r + G * (m + NW);
      if (j1 >= n) break;
      const bool two = j2 < n;
      const int j2c = two ? j2 : j1;
      const double vp1 = vprev[j1], wp1 = wprev[j1], vp2 = vprev[j2c], wp2 = wprev[j2c];
      double q1 = 0.0, q2 = 0.0;
      double* W1 = W + L * j1;
      double* W2 = W + L * j2c;
      int i = k + 1 + lane;
      // four rows per lane in flight: the column loads are issued before use
      for (; i + 96 < n; i += 128) {
        double a1[4], a2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a1[u] = W1[i + 32 * u];
          a2[u] = two ? W2[i + 32 * u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ii = i + 32 * u;
          const double vi = vprev[ii], wi = wprev[ii], ci = vcur[ii];
          a1[u] = fma(-wi, vp1, fma(-vi, wp1, a1[u]));
          q1 = fma(a1[u], ci, q1);
          if (two) {
            a2[u] = fma(-wi, vp2, fma(-vi, wp2, a2[u]));
            q2 = fma(a2[u], ci, q2);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          W1[i + 32 * u] = a1[u];
          if (two) W2[i + 32 * u] = a2[u];
        }
      }
      for (; i < n; i += 32) {
        const double vi = vprev[i], wi = wprev[i], ci = vcur[i];
        const double a1 = fma(-wi, vp1, fma(-vi, wp1, W1[i]));
        W1[i] = a1;
        q1 = fma(a1, ci, q1);
        if (two) {
          const double a2 = fma(-wi, vp2, fma(-vi, wp2, W2[i]));
          W2[i] = a2;
          q2 = fma(a2, ci, q2);
        }
        if (k == n - 2) d[n - 1] = a1;  // the last diagonal entry (i = j = n - 1)
      }
      q1 = t * warp_sum_xor(q1);
      q2 = t * warp_sum_xor(q2);
      if (lane == 0) {
        pk[j1] = q1;
        pv = fma(q1, vcur[j1], pv);
        if (two) {
          pk[j2] = q2;
          pv = fma(q2, vcur[j2], pv);
        }
      }
    }
    if (lane == 0) red[warp] = pv;
    __syncthreads();
    double* sdk = sdot + (k & 1) * (L / 2);
    if (tid == 0) {
      double sp = 0.0;
      for (int w = 0; w < NW; ++w) sp += red[w];
      sdk[r] = sp;
    }
    if (G > 1) {
      if (!trd_group_sync(bar, G * ++nb, s.err, &sh_ok)) return;
    } else {
      __syncthreads();
    }
    // w = p - (tau / 2) (p . v) v, kept with v for the next step's update
    if (warp == 0) {
      double sp = 0.0;
      for (int c = lane; c < G; c += 32) sp += __ldcg(&sdk[c]);
      sp = warp_sum_xor(sp);
      if (lane == 0) red[NW + 4] = 0.5 * t * sp;
    }
    for (int i = k + 1 + tid; i < n; i += kTrdNT) wprev[i] = __ldcg(&pk[i]);
    __syncthreads();
    const double half = red[NW + 4];
    for (int i = k + 1 + tid; i < n; i += kTrdNT) {
      wprev[i] = fma(-half, vcur[i], wprev[i]);
      vprev[i] = vcur[i];
    }
    __syncthreads();
  }
}

// The trailing update after panel q: A(k1:, k1:) -= V W^T + W V^T (rows and
// columns k1.., K = kPnb) on the tensor cores, as two FP64-accurate products
// whose operand rows are each all reflector entries or all W entries (one
// exponent per row then fits both, whatever the scale of C). Pack tiles: the
// 64-row blocks of V (first half of the tile range, sized for q = 0), then
// those of W.
int tiles_trd_s2k_pack(int n) { return n > kPnb ? 2 * (oz_rows_padded(n - kPnb) / 64) : 0; }
int tiles_trd_s2k(int n) { return n > kPnb ? ceil_div(n - kPnb, kOzBM) * ceil_div(n - kPnb, kOzBN) : 0; }

__global__ void __launch_bounds__(kOzNT) k_trd_s2k_pack(Search* S, TileMap tm, int q) {
  __shared__ int sh_e[64];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, k0 = kPnb * q, k1 = k0 + kPnb;
  if (k1 >= n) return;
  const int R = n - k1, half = oz_rows_padded(n - kPnb) / 64;
  const int which = tile >= half ? 1 : 0, rb = tile - which * half;
  if (rb >= oz_rows_padded(R) / 64) return;
  const TrdOz lay = trd_oz_layout(n);
  const long long L = s.ldn;
  const double* X = which == 0 ? s.EX + (k1 + L * k0) : s.EG + k1;  // V(k1 + i, l) or W(k1 + i, l)
  oz_pack_block_get([=] __device__(int i, int l) { return X[i + L * l]; }, false, R, kPnb, rb, oz_nks(kPnb),
                    s.ozp + (which == 0 ? lay.s2a : lay.s2b), s.oze + (which == 0 ? lay.ev : lay.ew), sh_e);
}

__global__ void __launch_bounds__(kOzNT, 1) k_trd_s2k(Search* S, TileMap tm, int q) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, k1 = kPnb * q + kPnb;
  if (k1 >= n) return;
  const int R = n - k1, TN = ceil_div(n - kPnb, kOzBN), mt = tile / TN, nt = tile % TN;
  if (mt * kOzBM >= R || nt * kOzBN >= R) return;
  const TrdOz lay = trd_oz_layout(n);
  const unsigned char* Vp = s.ozp + lay.s2a;
  const unsigned char* Wq8 = s.ozp + lay.s2b;
  const int* ev = s.oze + lay.ev;
  const int* ew = s.oze + lay.ew;
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long Wq[32];
  float Lq[32];
  const long long pitch = oz_pitch(oz_nks(kPnb));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = kOzBM * mt + 32 * (warp & 3) + lane, jb = kOzBN * nt + 32 * (warp >> 2);
  const long long L = s.ldn;
  double* Ai = s.EA + (k1 + i);
  bool ok = true;
  for (int part = 0; part < 2 && ok; ++part) {
    // part 0: V_i . W_j, part 1: W_i . V_j
    ok = oz_tile(cx, part == 0 ? Vp : Wq8, pitch, 2 * mt, part == 0 ? Wq8 : Vp, pitch, nt, oz_nks(kPnb), Wq, Lq);
    if (ok && i < R) {
      const int ei = part == 0 ? ev[i] : ew[i];
      const int* eb = part == 0 ? ew : ev;
#pragma unroll
      for (int qq = 0; qq < 32; ++qq) {
        const int jj = jb + qq;
        if (jj < R) Ai[L * (k1 + jj)] -= oz_value(Wq[qq], Lq[qq], ei, eb[jj]);
      }
    }
  }
  if (!ok && threadIdx.x == 0) atomicOr(s.err, kDevErrTimeout);
  oz_end(cx);
}

// --------------------------------------------------------------------------
// Scans of one CTA over n entries (n <= 4096): last index u <= t with
// flag(u) (prefix) or first index u >= t with flag(u) (suffix).
// --------------------------------------------------------------------------
template <int NT, class F>
__device__ void scan_last_start(int n, const F& flag, int* out, int* sh) {
  const int chunk = ceil_div(n, NT), c0 = threadIdx.x * chunk;
  int last = -1;
  for (int u = c0; u < c0 + chunk && u < n; ++u)
    if (flag(u)) last = u;
  sh[threadIdx.x] = last;
  __syncthreads();
  int carry = -1;
  for (int q = 0; q < static_cast<int>(threadIdx.x); ++q) carry = max(carry, sh[q]);
  for (int u = c0; u < c0 + chunk && u < n; ++u) {
    if (flag(u)) carry = u;
    out[u] = carry;
  }
  __syncthreads();
}

template <int NT, class F>
__device__ void scan_first_end(int n, const F& flag, int* out, int* sh) {
  const int chunk = ceil_div(n, NT), c0 = threadIdx.x * chunk;
  int first = 0x7fffffff;
  for (int u = min(c0 + chunk, n) - 1; u >= c0; --u)
    if (flag(u)) first = u;
  sh[threadIdx.x] = first;
  __syncthreads();
  int carry = 0x7fffffff;
  for (int q = NT - 1; q > static_cast<int>(threadIdx.x); --q) carry = min(carry, sh[q]);
  for (int u = min(c0 + chunk, n) - 1; u >= c0; --u) {
    if (flag(u)) carry = u;
    out[u] = carry + 1;  // block end (exclusive)
  }
  __syncthreads();
}

// --------------------------------------------------------------------------
// 2. ||T|| bound, splitting and the blocks of T (one CTA per search).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrdNT) k_trd_blocks(Search* S, int s0) {
  __shared__ double red[32];
  __shared__ int shi[kTrdNT];
  Search& s = S[s0 + blockIdx.x];
  if (!trd_due(s)) return;
  const int n = s.n;
  const double* d = tv(s, TV_D);
  const double* e = tv(s, TV_E);
  double* es = tv(s, TV_ES);
  double* e2 = tv(s, TV_E2);
  double* sc = tv(s, TV_SCAL);
  double tn = 0.0, em = 0.0;
  for (int i = threadIdx.x; i < n; i += kTrdNT) {
    const double lo = i > 0 ? fabs(e[i - 1]) : 0.0, hi = i + 1 < n ? fabs(e[i]) : 0.0;
    tn = fmax(tn, fabs(d[i]) + lo + hi);
    em = fmax(em, hi);
  }
  tn = block_max<kTrdNT>(tn, red);
  em = block_max<kTrdNT>(em, red);
  const double split = kTrdSplit * sqrt(static_cast<double>(n)) * kTrdEps * tn;
  for (int i = threadIdx.x; i + 1 < n; i += kTrdNT) {
    const double x = fabs(e[i]) <= split ? 0.0 : e[i];
    es[i] = x;
    e2[i] = x * x;
  }
  // d and e^2 scaled by a power of two (|d| <= 1) in FP32 for the first
  // bisection steps (the reduction's buffers TV_P0 and TV_P1 are free now)
  const double scl = tn > 0.0 ? exp2(-static_cast<double>(ilogb(tn) + 1)) : 1.0;
  // as pairs hi + lo of floats (hi the rounded value, lo the rounded rest):
  // d at TV_P0 (hi, then lo from ldn on), e^2 at TV_P1 likewise
  float* d32 = reinterpret_cast<float*>(tv(s, TV_P0));
  float* e32 = reinterpret_cast<float*>(tv(s, TV_P1));
  const long long L2 = s.ldn;
  for (int i = threadIdx.x; i < n; i += kTrdNT) {
    const double ds = d[i] * scl;
    d32[i] = static_cast<float>(ds);
    d32[L2 + i] = static_cast<float>(ds - static_cast<double>(d32[i]));
    if (i + 1 < n) {
      const double x = fabs(e[i]) <= split ? 0.0 : e[i] * scl;
      const double x2 = x * x;
      e32[i] = static_cast<float>(x2);
      e32[L2 + i] = static_cast<float>(x2 - static_cast<double>(e32[i]));
    }
  }
  if (threadIdx.x == 0) {
    sc[7] = scl;
    sc[0] = tn;
    sc[1] = DBL_MIN * fmax(1.0, em * em);
    sc[2] = split;
    sc[3] = kTrdClus * tn;
    sc[4] = 0.0;  // orthogonality defects before the Newton-Schulz steps
    sc[5] = 0.0;
    sc[6] = 0.0;
  }
  __syncthreads();
  int* b0 = ti(s, TI_B0);
  int* b1 = ti(s, TI_B1);
  scan_last_start<kTrdNT>(n, [&](int u) { return u == 0 || es[u - 1] == 0.0; }, b0, shi);
  scan_first_end<kTrdNT>(n, [&](int u) { return u == n - 1 || es[u] == 0.0; }, b1, shi);
}

// --------------------------------------------------------------------------
// 3. Multisection: a group of LANES lanes finds eigenvalue t - b0 (ascending)
// of its block; each round the lanes take the Sturm counts at LANES interior
// points of the bracket, which shrinks it (LANES + 1)-fold. Eight lanes cut the
// sequential rounds from ~52 to ~17 for the few eigenvalues of one search; a
// large batch, which fills the GPU with eigenvalues anyway, takes one lane
// (plain bisection: the fewest counts in total). The counts' reciprocals come
// from an FP32 estimate and two Newton steps in FP64 (exact to rounding)
// instead of an FP64 divide.
// --------------------------------------------------------------------------
constexpr int kTrdTT = 128;   // threads per tile of the per-eigenvalue kernels
constexpr int kTrdBisLanes = 8;
int tiles_trd(int n) { return ceil_div(n, kTrdTT); }
int tiles_trd_bis(int n) { return ceil_div(n * kTrdBisLanes, kTrdTT); }

// 1 / q from the FP32 reciprocal and two Newton steps inside 2^-99 < |q| <
// 2^99 (exponent tested on the integer pattern), the division elsewhere.
__device__ __forceinline__ double fast_rcp(double q) {
  const int ex = (__double2hiint(q) >> 20) & 0x7FF;
  if (ex > 1023 - 99 && ex < 1023 + 99) {
    double r = static_cast<double>(__frcp_rn(static_cast<float>(q)));
    r = r * fma(-q, r, 2.0);
    return r * fma(-q, r, 2.0);
  }
  return 1.0 / q;
}

// Sturm count: eigenvalues of block [b0, b1) below x (pivots of magnitude at
// most pivmin replaced by -pivmin; |q| and pivmin compared as ordered bit
// patterns, the sign read from the sign bit).
__device__ __forceinline__ int sturm64(const double* d, const double* e2, int b0, int b1, double x, double pivmin) {
  const long long pb = __double_as_longlong(pivmin);
  int cnt = 0;
  double qq = d[b0] - x;
  if ((__double_as_longlong(qq) & 0x7FFFFFFFFFFFFFFFLL) <= pb) qq = -pivmin;
  cnt += static_cast<int>(static_cast<unsigned long long>(__double_as_longlong(qq)) >> 63);
  for (int j = b0 + 1; j < b1; ++j) {
    qq = (d[j] - x) - e2[j - 1] * fast_rcp(qq);
    if ((__double_as_longlong(qq) & 0x7FFFFFFFFFFFFFFFLL) <= pb) qq = -pivmin;
    cnt += static_cast<int>(static_cast<unsigned long long>(__double_as_longlong(qq)) >> 63);
  }
  return cnt;
}

// The same in FP32 on the scaled copies (|d| <= 1).
__device__ __forceinline__ int sturm32(const float* d, const float* e2, int b0, int b1, float x) {
  constexpr float piv = 0x1p-90f;
  int cnt = 0;
  float qq = d[b0] - x;
  if (fabsf(qq) <= piv) qq = -piv;
  cnt += qq < 0.0f;
  for (int j = b0 + 1; j < b1; ++j) {
    qq = (d[j] - x) - e2[j - 1] * __frcp_rn(qq);
    if (fabsf(qq) <= piv) qq = -piv;
    cnt += qq < 0.0f;
  }
  return cnt;
}

// The same in double-float arithmetic (each value a pair hi + lo of floats,
// ~48 significant bits; error-free sums and products from FMA) on the scaled
// pairs: d at d32 / d32 + ldn, e^2 at e32 / e32 + ldn, x = xh + xl.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ int sturm_df(const float* dh, const float* dl, const float* eh, const float* el,
                                        int b0, int b1, float xh, float xl) {
  constexpr float piv = 0x1p-90f;
  int cnt = 0;
  float qh, ql;
  {
    float s, e;
    df_two_sum(dh[b0], -xh, s, e);
    e = __fadd_rn(e, __fsub_rn(dl[b0], xl));
    qh = __fadd_rn(s, e);
    ql = __fsub_rn(e, __fsub_rn(qh, s));
  }
  if (fabsf(qh) <= piv) {
    qh = -piv;
    ql = 0.0f;
  }
  cnt += qh < 0.0f;
  for (int j = b0 + 1; j < b1; ++j) {
    // t = d_j - x
    float th, tl;
    {
      float s, e;
      df_two_sum(dh[j], -xh, s, e);
      e = __fadd_rn(e, __fsub_rn(dl[j], xl));
      th = __fadd_rn(s, e);
      tl = __fsub_rn(e, __fsub_rn(th, s));
    }
    // u = e2 / q: leading quotient, then the rest from the exact residual
    const float e2h = eh[j - 1], e2l = el[j - 1];
    const float uh = __fdiv_rn(e2h, qh);
    const float p = __fmul_rn(uh, qh);
    const float pe = __fmaf_rn(uh, qh, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(e2h, p), pe), __fmaf_rn(-uh, ql, e2l));
    const float ul = __fdiv_rn(r, qh);
    // q = t - u
    float s, e;
    df_two_sum(th, -uh, s, e);
    e = __fadd_rn(e, __fsub_rn(tl, ul));
    qh = __fadd_rn(s, e);
    ql = __fsub_rn(e, __fsub_rn(qh, s));
    if (fabsf(qh) <= piv) {
      qh = -piv;
      ql = 0.0f;
    }
    cnt += qh < 0.0f;
  }
  return cnt;
}

// Eigenvalue t of its block by bisection (LANES = 1) or multisection with
// LANES points per step, in three precisions: FP32 on the scaled block down to
// a width of 2^-19 ||T||, widened by 2^-18 ||T|| (eight times the backward
// error of an FP32 Sturm count, ~10 eps32 ||T||); double-float down to
// 2^-43 ||T||, widened by 2^-42 ||T|| (six times that of a double-float
// count, ~10 2^-48 ||T||); each widened bracket checked with two counts of
// the next precision (the previous bracket kept if the check fails), the
// last step in FP64 to 4 eps64 ||T||. The FP64 counts are the bulk of the
// work (the FP64 pipe is ~80 % busy), so every precision goes as far as its
// counts stay reliable.
template <int LANES>
__global__ void __launch_bounds__(kTrdTT) k_trd_bisect(Search* S, TileMap tm) {
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n;
  const int q = threadIdx.x % LANES;
  const int t = tile * (kTrdTT / LANES) + threadIdx.x / LANES;
  if (t >= n) return;  // uniform across the lanes of a group
  const int base = (threadIdx.x & 31) & ~(LANES - 1);
  const unsigned gmask = static_cast<unsigned>((1ull << LANES) - 1) << base;
  const double* d = tv(s, TV_D);
  const double* es = tv(s, TV_ES);
  const double* e2 = tv(s, TV_E2);
  const float* d32 = reinterpret_cast<const float*>(tv(s, TV_P0));
  const float* e32 = reinterpret_cast<const float*>(tv(s, TV_P1));
  const double* sc = tv(s, TV_SCAL);
  double* lamb = tv(s, TV_LAMB);
  const int b0 = ti(s, TI_B0)[t], b1 = ti(s, TI_B1)[t];
  if (b1 - b0 == 1) {
    if (q == 0) lamb[t] = d[t];
    return;
  }
  // the start bracket: [-||T||, ||T||] with ||T|| the largest Gershgorin row
  // sum of the unsplit T (it holds every block's spectrum), widened for rounding
  const double tn = sc[0], pivmin = sc[1], scl = sc[7];
  const double atol = 4.0 * kTrdEps * tn;
  const double fudge = 2.0 * kTrdEps * tn * (b1 - b0) + 2.0 * pivmin;
  double lo = -tn - fudge, hi = tn + fudge;
  const int idx = t - b0;
  // one multisection step on [lo, hi] from the counts of the LANES points
  auto narrow = [&](auto& lo_, auto& hi_, int cnt, auto w) -> bool {
    const unsigned le = __ballot_sync(gmask, cnt <= idx) & gmask;
    const int qlo = le ? (31 - __clz(le)) - base : -1;
    const auto nlo = qlo >= 0 ? lo_ + w * (qlo + 1) : lo_;
    const auto nhi = qlo + 1 < LANES ? lo_ + w * (qlo + 2) : hi_;
    if (!(nlo < nhi) || (nlo == lo_ && nhi == hi_)) return false;
    lo_ = nlo;
    hi_ = nhi;
    return true;
  };
  // the two ends of a candidate bracket checked by the counts `cnt` (lane 0
  // the left end, lane 1 the right one; one lane does both)
  auto check = [&](auto cnt, double a, double b) -> bool {
    if (LANES == 1) return cnt(a) <= idx && cnt(b) > idx;
    bool mine = true;
    if (q == 0) mine = cnt(a) <= idx;
    if (q == 1) mine = cnt(b) > idx;
    return (__ballot_sync(gmask, !mine) & gmask) == 0;
  };
  if (tn > 0.0) {
    const long long L2 = s.ldn;
    // FP32
    float lo32 = static_cast<float>(lo * scl), hi32 = static_cast<float>(hi * scl);
    for (int it = 0; it < 40 && hi32 - lo32 > 0x1p-19f; ++it) {
      const float w = (hi32 - lo32) / (LANES + 1);
      if (!narrow(lo32, hi32, sturm32(d32, e32, b0, b1, lo32 + w * (q + 1)), w)) break;
    }
    auto cnt_df = [&](double xs) {  // x given scaled, in FP64
      const float xh = static_cast<float>(xs);
      return sturm_df(d32, d32 + L2, e32, e32 + L2, b0, b1, xh, static_cast<float>(xs - static_cast<double>(xh)));
    };
    double los = lo * scl, his = hi * scl;  // scaled bracket, FP64
    {
      const double a = fmax(los, static_cast<double>(lo32) - 0x1p-18), b = fmin(his, static_cast<double>(hi32) + 0x1p-18);
      if (a < b && check(cnt_df, a, b)) {
        los = a;
        his = b;
      }
    }
    // double-float
    for (int it = 0; it < 60 && his - los > 0x1p-43; ++it) {
      const double w = (his - los) / (LANES + 1);
      if (!narrow(los, his, cnt_df(los + w * (q + 1)), w)) break;
    }
    const double lo2 = fmax(lo, (los - 0x1p-42) / scl), hi2 = fmin(hi, (his + 0x1p-42) / scl);
    if (lo2 < hi2 && check([&](double x) { return sturm64(d, e2, b0, b1, x, pivmin); }, lo2, hi2)) {
      lo = lo2;
      hi = hi2;
    }
  }
  for (int it = 0; it < 160 && hi - lo > atol; ++it) {
    const double w = (hi - lo) / (LANES + 1);
    if (!narrow(lo, hi, sturm64(d, e2, b0, b1, lo + w * (q + 1), pivmin), w)) break;
  }
  if (q == 0) lamb[t] = 0.5 * (lo + hi);
}

// --------------------------------------------------------------------------
// 4a. Ranks of the eigenvalues (ascending, ties by block-major index) and the
// clusters of close eigenvalues within a block (one CTA per search).
// --------------------------------------------------------------------------
constexpr int kTrdSortNT = 1024;

__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

__global__ void __launch_bounds__(kTrdSortNT) k_trd_rank(Search* S, int s0) {
  __shared__ int shi[kTrdSortNT];
  Search& s = S[s0 + blockIdx.x];
  if (!trd_due(s)) return;
  const int n = s.n;
  const double* lamb = tv(s, TV_LAMB);
  double* lams = tv(s, TV_LAMS);
  int* rank = ti(s, TI_RANK);
  const int* b0 = ti(s, TI_B0);
  const double ctol = tv(s, TV_SCAL)[3];
  for (int t = threadIdx.x; t < n; t += kTrdSortNT) {
    const long long kt = order_key(lamb[t]);
    int r = 0;
    for (int u = 0; u < n; ++u) {
      const long long ku = order_key(lamb[u]);
      r += (ku < kt) || (ku == kt && u < t);
    }
    rank[t] = r;
    lams[r] = lamb[t];
  }
  scan_last_start<kTrdSortNT>(
      n, [&](int u) { return u == b0[u] || !(lamb[u] - lamb[u - 1] <= ctol); }, ti(s, TI_CL0), shi);
}

// --------------------------------------------------------------------------
// 4b. Inverse iteration (thread t, eigenvalue lamb[t] of its block): three
// solves of (T - lambda I) x = x_prev with one Gaussian elimination with
// partial pivoting (its factors in scratch interleaved by thread), the
// iterate in column t of ET.
// --------------------------------------------------------------------------
__device__ __forceinline__ double start_value(int t, int j) {
  uint32_t h = static_cast<uint32_t>(t) * 0x9E3779B1u ^ (static_cast<uint32_t>(j) * 0x85EBCA77u);
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (static_cast<double>(h) + 0.5) * 0x1p-31 - 1.0;  // in (-1, 1)
}

constexpr long long kInvitSwap = 0x7ff8000000000000LL;  // a quiet NaN: the row-interchange flag

__global__ void __launch_bounds__(kTrdTT) k_trd_invit(Search* S, TileMap tm) {
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, t = tile * kTrdTT + threadIdx.x;
  if (t >= n) return;
  const long long L = s.ldn, nn = n;
  const double* d = tv(s, TV_D);
  const double* es = tv(s, TV_ES);
  const double lam = tv(s, TV_LAMB)[t];
  const double tiny = kTrdEps * tv(s, TV_SCAL)[0];
  const int b0 = ti(s, TI_B0)[t], b1 = ti(s, TI_B1)[t];
  double* x = s.ET + L * t;
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  if (b1 - b0 == 1) {
    x[t] = 1.0;
    return;
  }
  double* u0 = s.EA;
  double* u1 = s.EG;
  double* u2 = s.EH;
  auto piv_of = [&](double a) { return fabs(a) > tiny ? a : (a < 0.0 ? -tiny : tiny); };
  // factorisation of T - lambda I, once for the three solves: row j without
  // an interchange keeps 1 / pivot (u0), its superdiagonal (u1) and the
  // multiplier (u2); a row with one keeps the multiplier (u0) and the flag
  // kInvitSwap in u1 (its U row, e_j, d_{j+1} - lambda, e_{j+1}, is read from
  // T again when it is needed)
  double a = d[b0] - lam, b = es[b0], c = 0.0;
  for (int j = b0; j + 1 < b1; ++j) {
    const double sub = es[j], nd = d[j + 1] - lam, nsup = (j + 2 < b1) ? es[j + 1] : 0.0;
    const long long o = j * nn + t;
    if (fabs(a) >= fabs(sub)) {
      const double r = 1.0 / piv_of(a);
      const double l = sub * r;
      u0[o] = r;
      u1[o] = b;
      u2[o] = l;
      a = nd - l * b;
      b = nsup - l * c;
    } else {
      const double l = a / sub;
      u0[o] = l;
      u1[o] = __longlong_as_double(kInvitSwap);
      const double a2 = b - l * nd;
      b = c - l * nsup;
      a = a2;
    }
    c = 0.0;
  }
  const double rlast = 1.0 / piv_of(a);
  for (int j = b0; j < b1; ++j) x[j] = start_value(t, j);
  for (int it = 0; it < 3; ++it) {
    // forward: the same row interchanges and multipliers on the iterate
    double y = x[b0];
    for (int j = b0; j + 1 < b1; ++j) {
      const long long o = j * nn + t;
      const double yn = x[j + 1];
      if (__double_as_longlong(u1[o]) != kInvitSwap) {
        x[j] = y;
        y = yn - u2[o] * y;
      } else {
        x[j] = yn;
        y = y - u0[o] * yn;
      }
    }
    // back substitution, then normalise
    double xn1 = y * rlast, xn2 = 0.0;
    x[b1 - 1] = xn1;
    double ss = xn1 * xn1;
    for (int j = b1 - 2; j >= b0; --j) {
      const long long o = j * nn + t;
      const double ub = u1[o];
      double v;
      if (__double_as_longlong(ub) != kInvitSwap) {
        v = (x[j] - ub * xn1) * u0[o];
      } else {
        const double nd = d[j + 1] - lam, nsup = (j + 2 < b1) ? es[j + 1] : 0.0;
        v = (x[j] - nd * xn1 - nsup * xn2) / es[j];
      }
      x[j] = v;
      xn2 = xn1;
      xn1 = v;
      ss = fma(v, v, ss);
    }
    const double inv = 1.0 / sqrt(ss);
    for (int j = b0; j < b1; ++j) x[j] *= inv;
  }
}

// --------------------------------------------------------------------------
// 4c. Gram-Schmidt (twice) inside each cluster of close eigenvalues of one
// block, in chunks of at most kTrdClusMax consecutive vectors (independent of
// one another). A long chunk on a long block goes to a whole CTA as classical
// Gram-Schmidt applied twice (all projections of a vector at once: the dots
// spread over the warps, the update over the rows, the vector in shared
// memory); a short one to one warp as modified Gram-Schmidt, twice. Both keep
// the orthogonality that the later Newton-Schulz steps need (Giraud, Langou &
// Rozloznik 2005: two passes of either are enough for vectors that are not
// numerically dependent).
// --------------------------------------------------------------------------
// Modified Gram-Schmidt, twice, on vectors [c, ce) of rows [r0, r1) (one warp).
__device__ void cluster_mgs(double* V, long long L, int c, int ce, int r0, int r1, int lane) {
  double* vc = V + L * c;
  {
    double q = 0.0;
    for (int i = r0 + lane; i < r1; i += 32) q = fma(vc[i], vc[i], q);
    const double inv = 1.0 / sqrt(warp_sum_xor(q));
    for (int i = r0 + lane; i < r1; i += 32) vc[i] *= inv;
    __syncwarp();
  }
  for (int a = c + 1; a < ce; ++a) {
    double* va = V + L * a;
    for (int rep = 0; rep < 2; ++rep)
      for (int b = c; b < a; ++b) {
        const double* vb = V + L * b;
        double p = 0.0;
        for (int i = r0 + lane; i < r1; i += 32) p = fma(vb[i], va[i], p);
        p = warp_sum_xor(p);
        for (int i = r0 + lane; i < r1; i += 32) va[i] = fma(-p, vb[i], va[i]);
        __syncwarp();
      }
    double q = 0.0;
    for (int i = r0 + lane; i < r1; i += 32) q = fma(va[i], va[i], q);
    const double inv = 1.0 / sqrt(warp_sum_xor(q));
    for (int i = r0 + lane; i < r1; i += 32) va[i] *= inv;
    __syncwarp();
  }
}

// Classical Gram-Schmidt, twice, on vectors [c, ce) of rows [r0, r1) (the
// whole CTA; r1 - r0 <= kEigBigMaxN). Per vector a and pass: p = V_prev^T v_a
// (warp w takes the previous vectors w, w + 8, ...), then v_a -= V_prev p on
// every row (the terms in ascending order); then v_a / |v_a|.
__device__ void cluster_cgs2_cta(double* V, long long L, int c, int ce, int r0, int r1, double* va,
                                 double* pb, double* red) {
  constexpr int NW = kTrdNT / 32;
  const int R = r1 - r0, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int a = c; a < ce; ++a) {
    double* col = V + L * a + r0;
    for (int i = tid; i < R; i += kTrdNT) va[i] = col[i];
    __syncthreads();
    const int m = a - c;
    for (int rep = 0; rep < (m > 0 ? 2 : 0); ++rep) {
      for (int x = warp; x < m; x += NW) {
        const double* vb = V + L * (c + x) + r0;
        double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
        int i = lane;
        for (; i + 96 < R; i += 128) {  // four rows per lane in flight
          p0 = fma(vb[i], va[i], p0);
          p1 = fma(vb[i + 32], va[i + 32], p1);
          p2 = fma(vb[i + 64], va[i + 64], p2);
          p3 = fma(vb[i + 96], va[i + 96], p3);
        }
        for (; i < R; i += 32) p0 = fma(vb[i], va[i], p0);
        const double p = warp_sum_xor((p0 + p1) + (p2 + p3));
        if (lane == 0) pb[x] = p;
      }
      __syncthreads();
      for (int i = tid; i < R; i += kTrdNT) {
        const double* vb = V + L * c + r0 + i;
        double acc = va[i];
        int x = 0;
        for (; x + 4 <= m; x += 4) {
          const double b0 = vb[L * x], b1 = vb[L * (x + 1)], b2 = vb[L * (x + 2)], b3 = vb[L * (x + 3)];
          acc = fma(-pb[x], b0, acc);
          acc = fma(-pb[x + 1], b1, acc);
          acc = fma(-pb[x + 2], b2, acc);
          acc = fma(-pb[x + 3], b3, acc);
        }
        for (; x < m; ++x) acc = fma(-pb[x], vb[L * x], acc);
        va[i] = acc;
      }
      __syncthreads();
    }
    double q = 0.0;
    for (int i = tid; i < R; i += kTrdNT) q = fma(va[i], va[i], q);
    q = warp_sum_xor(q);
    if (lane == 0) red[warp] = q;
    __syncthreads();
    double nq = 0.0;
    for (int w = 0; w < NW; ++w) nq += red[w];
    const double inv = 1.0 / sqrt(nq);
    for (int i = tid; i < R; i += kTrdNT) col[i] = va[i] * inv;
    __syncthreads();  // v_a complete before the next vector reads it (and red is reused)
  }
}

constexpr int kTrdMgsCtas = 32;    // CTAs per search of the Gram-Schmidt kernel
constexpr int kTrdCgsMinVec = 8;   // chunks of at least this many vectors
constexpr int kTrdCgsMinRows = 256;  // on blocks of at least this many rows go to a CTA

__global__ void __launch_bounds__(kTrdNT) k_trd_mgs(Search* S, int s0) {
  __shared__ double va[kEigBigMaxN];
  __shared__ double pb[kTrdClusMax];
  __shared__ double red[kTrdNT / 32];
  Search& s = S[s0 + blockIdx.x];
  if (!trd_due(s)) return;
  const int n = s.n, lane = threadIdx.x & 31;
  const int warp = blockIdx.y * (kTrdNT / 32) + (threadIdx.x >> 5);  // of the search's warps
  const long long L = s.ldn;
  const int* cl0 = ti(s, TI_CL0);
  const int* b0a = ti(s, TI_B0);
  const int* b1a = ti(s, TI_B1);
  double* V = s.ET;
  // work items: the chunks of every cluster of two or more; the long ones
  // dealt round-robin to the CTAs (pass 0), the others to the warps (pass 1)
  for (int pass = 0; pass < 2; ++pass) {
    int found = 0;
    for (int c = 0; c < n; ++c) {
      if (cl0[c] != c || c + 1 >= n || cl0[c + 1] != c) continue;
      int ce = c + 1;
      while (ce < n && cl0[ce] == c) ++ce;
      const int r0 = b0a[c], r1 = b1a[c];
      for (int cc = c; cc < ce; cc += kTrdClusMax) {
        const int cn = min(ce, cc + kTrdClusMax);
        const bool big = cn - cc >= kTrdCgsMinVec && r1 - r0 >= kTrdCgsMinRows;
        if (big != (pass == 0)) continue;
        if (big) {
          if ((found++ % kTrdMgsCtas) == static_cast<int>(blockIdx.y))
            cluster_cgs2_cta(V, L, cc, cn, r0, r1, va, pb, red);
        } else if ((found++ % (kTrdMgsCtas * kTrdNT / 32)) == warp) {
          cluster_mgs(V, L, cc, cn, r0, r1, lane);
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// 5. Newton-Schulz: M = (I - V^T V) / 2 in FP32 from an FP64-accurate
// product on the tensor cores (64 x 64 tiles, mirrored; tiles outside the
// eigenvalue band are zero and flagged so), then V' = V + V M with FP32
// products over the nonzero tiles.
// --------------------------------------------------------------------------
int tiles_trd_sq(int n) { const int T = ceil_div(n, kGBM); return T * T; }

int tiles_trd_ozp(int n) { return oz_rows_padded(n) / 64; }
int tiles_trd_ozg(int n) { return ceil_div(n, kOzBM) * ceil_div(n, kOzBN); }
size_t trd_oz_bytes(int n) { return trd_oz_layout(n).total; }
int trd_oz_exps(int n) { return trd_oz_layout(n).etotal; }

__device__ __forceinline__ bool trd_ns_skipped(const Search& s, int pass) {
  return pass > 0 && __ldcg(&tv(s, TV_SCAL)[3 + pass]) <= kTrdNsSkip;  // the previous step was enough
}

// The columns of this pass's V as the rows of a packed operand (K = n).
__global__ void __launch_bounds__(kOzNT) k_trd_oz_pack(Search* S, TileMap tm, int pass) {
  __shared__ int sh_e[64];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s) || trd_ns_skipped(s, pass)) return;
  const double* V = (pass & 1) ? s.EA : s.ET;
  oz_pack_block(V, s.ldn, 1, s.n, s.n, tile, oz_nks(s.n), s.ozp, s.oze, sh_e);
}

// M = (I - V^T V) / 2 over the 64 x 64 tiles (fi, fj), fi <= fj, that hold a
// pair of one block with eigenvalues within kTrdNsBand ||T|| (mirrored,
// flagged; zero and unflagged elsewhere), from the FP64-accurate tensor-core
// product: CTA (bi, bj) owns the 128 x 64 tile of rows 128 bi.., columns
// 64 bj.., i.e. the 64 x 64 tiles (2 bi, bj) and (2 bi + 1, bj), and writes
// the elements i <= j of those it owns.
__global__ void __launch_bounds__(kOzNT, 1) k_trd_oz_gram(Search* S, TileMap tm, int pass) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  __shared__ double trange[3][2];
  __shared__ int brange[3][2];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s) || trd_ns_skipped(s, pass)) return;
  const int n = s.n, T = ceil_div(n, kGBM), TN = ceil_div(n, kOzBN);
  const int bi = tile / TN, bj = tile % TN;
  if (bj * kOzBN + kOzBN - 1 < bi * kOzBM) return;  // wholly below the diagonal
  const long long L = s.ldn;
  float* M = reinterpret_cast<float*>(s.EG);
  int* flags = ti(s, TI_TFLAG);
  double* sc = tv(s, TV_SCAL);
  // eigenvalue and block ranges of the column blocks 2 bi, 2 bi + 1 and bj
  if (threadIdx.x < 96) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int c0 = (w == 0 ? 2 * bi : (w == 1 ? 2 * bi + 1 : bj)) * kGBM;
    double lo = INFINITY, hi = -INFINITY;
    int blo = 0x7fffffff, bhi = -1;
    for (int u = l; u < kGBM; u += 32) {
      const int t = c0 + u;
      if (t < n) {
        const double lam = tv(s, TV_LAMB)[t];
        const int b = ti(s, TI_B0)[t];
        lo = fmin(lo, lam);
        hi = fmax(hi, lam);
        blo = min(blo, b);
        bhi = max(bhi, b);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      blo = min(blo, __shfl_xor_sync(0xffffffffu, blo, o));
      bhi = max(bhi, __shfl_xor_sync(0xffffffffu, bhi, o));
    }
    if (l == 0) {
      trange[w][0] = lo;
      trange[w][1] = hi;
      brange[w][0] = blo;
      brange[w][1] = bhi;
    }
  }
  __syncthreads();
  bool owned[2], needed[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int fi = 2 * bi + h;
    owned[h] = fi <= bj && fi < T;
    const bool share = brange[h][0] <= brange[2][1] && brange[2][0] <= brange[h][1];
    const double dist = fmax(0.0, fmax(trange[2][0] - trange[h][1], trange[h][0] - trange[2][1]));
    needed[h] = owned[h] && share && !(dist > kTrdNsBand * sc[0]);
    if (owned[h] && threadIdx.x == 0) {
      flags[fi + T * bj] = needed[h];
      flags[bj + T * fi] = needed[h];
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = bi * kOzBM + 32 * (warp & 3) + lane;
  const int h = (warp & 3) >> 1;
  const int jb = bj * kOzBN + 32 * (warp >> 2);
  if (!needed[0] && !needed[1]) {  // M = 0 on the owned tiles and their mirrors
    if (owned[h] && i < n)
      for (int q = 0; q < 32; ++q) {
        const int j = jb + q;
        if (j < n && i <= j) {
          M[i + L * j] = 0.f;
          M[j + L * i] = 0.f;
        }
      }
    return;
  }
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long Wq[32];
  float Lq[32];
  const long long pitch = oz_pitch(oz_nks(n));
  const bool ok = oz_tile(cx, s.ozp, pitch, 2 * bi, s.ozp, pitch, bj, oz_nks(n), Wq, Lq);
  double dmax = 0.0;
  if (ok && owned[h] && i < n) {
    const int ei = s.oze[i];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int j = jb + q;
      if (j < n && i <= j) {
        double m = 0.0;
        if (needed[h]) {
          const int ej = s.oze[j];
          const double g = oz_value(Wq[q], Lq[q], ei, ej);
          m = 0.5 * ((i == j ? 1.0 : 0.0) - g);
          dmax = fmax(dmax, fabs(m));
        }
        M[i + L * j] = static_cast<float>(m);
        M[j + L * i] = static_cast<float>(m);
      }
    }
  }
  // the defect of this pass (non-negative doubles order like their bit
  // patterns); every lane of every warp takes part in the reduction
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (lane == 0 && dmax > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&sc[4 + pass]),
              static_cast<unsigned long long>(__double_as_longlong(dmax)));
  if (!ok && threadIdx.x == 0) atomicOr(s.err, kDevErrTimeout);
  oz_end(cx);
}

struct GemmSmem32 {
  float As[kGBK][kGBM];
  float Bs[kGBK][kGBN];
};

// Step `pass` (0, 1, 2) maps ET -> EA, EA -> ET, ET -> EA: V' = V + V M, or a
// copy when the previous step started from a defect small enough (then no M
// was formed); the result is in EA after the three.
// V' = V + V M on one 64 x 64 tile of V': 256 threads, each a 4 x 4 block of
// consecutive rows and columns (float4 reads of the staged operands), k in
// steps of 32 over the k tiles whose 64 x 64 block of M is flagged nonzero,
// the next step's operands loaded into registers while the current one is
// multiplied (two shared-memory buffers, one barrier per step). The products
// are summed in ascending k, one FP32 FMA each.
constexpr int kNsBK = 32;

__global__ void __launch_bounds__(kGNT) k_trd_ns(Search* S, TileMap tm, int pass) {
  __shared__ __align__(16) float As[2][kNsBK][kGBM];      // V block, [k][i]
  __shared__ __align__(16) float Bs[2][kNsBK][kGBN + 4];  // M block, [k][j] (rows 16-byte aligned)
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, T = ceil_div(n, kGBM);
  const int i0 = (tile % T) * kGBM, j0 = (tile / T) * kGBN;
  const long long L = s.ldn;
  const double* V = (pass & 1) ? s.EA : s.ET;
  double* Vo = (pass & 1) ? s.ET : s.EA;
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  if (pass > 0 && __ldcg(&tv(s, TV_SCAL)[3 + pass]) <= kTrdNsSkip) {
    for (int e = tid; e < kGBM * kGBN; e += kGNT) {
      const int i = i0 + (e & (kGBM - 1)), j = j0 + e / kGBM;
      if (i < n && j < n) Vo[i + L * j] = V[i + L * j];
    }
    return;
  }
  const float* M = reinterpret_cast<const float*>(s.EG);
  const int* flags = ti(s, TI_TFLAG);
  const int nkt = ceil_div(n, kNsBK);
  auto next_kt = [&](int kt) {  // the first k step at or after kt on a flagged block of M
    while (kt < nkt && !__ldcg(&flags[(kt * kNsBK) / kGBM + T * (j0 / kGBN)])) ++kt;
    return kt;
  };
  float ra[8], rb[8];
  auto load = [&](int kt) {
    const int k0 = kt * kNsBK;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * kGNT;
      const int ii = e & (kGBM - 1), kk = e >> 6;  // V: consecutive threads, consecutive rows
      const int gi = i0 + ii, gk = k0 + kk;
      ra[q] = (gi < n && gk < n) ? static_cast<float>(V[gi + L * gk]) : 0.f;
      const int kk2 = e & (kNsBK - 1), jj = e >> 5;  // M: consecutive threads, consecutive k
      const int gk2 = k0 + kk2, gj = j0 + jj;
      rb[q] = (gk2 < n && gj < n) ? M[gk2 + L * gj] : 0.f;
    }
  };
  auto store = [&](int b) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * kGNT;
      As[b][e >> 6][e & (kGBM - 1)] = ra[q];
      Bs[b][e & (kNsBK - 1)][e >> 5] = rb[q];
    }
  };
  float acc[4][4] = {};
  int kt = next_kt(0);
  if (kt < nkt) {
    load(kt);
    store(0);
  }
  __syncthreads();
  int b = 0;
  while (kt < nkt) {
    const int kn = next_kt(kt + 1);
    if (kn < nkt) load(kn);
#pragma unroll 8
    for (int kk = 0; kk < kNsBK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[b][kk][4 * tr]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[b][kk][4 * tc]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    if (kn < nkt) store(b ^ 1);
    __syncthreads();
    b ^= 1;
    kt = kn;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + 4 * tr + r, j = j0 + 4 * tc + c;
      if (i < n && j < n) Vo[i + L * j] = V[i + L * j] + static_cast<double>(acc[r][c]);
    }
}

// --------------------------------------------------------------------------
// 6. Back-transformation B = Q V' of the smaller sizes (reflectors applied in
// reverse order, one warp per column), canonical sign, and the column order of
// ascending eigenvalues; kernels_eig_trd_bt.cu takes n >= kBtBlockedMinN.
// --------------------------------------------------------------------------
__host__ __device__ inline int trd_bt_cols(int n) { return 8; }
int tiles_trd_bt(int n) { return trd_bt_blocked(n) ? 0 : ceil_div(n, trd_bt_cols(n)); }

// Each column held in registers (element lane + 32 r in x[r]; n <= 32 RMAX):
// the column never moves; each reflector is staged once
// per CTA in shared memory (double-buffered: the next one is loaded while the
// current one is applied) and rows at or above its first row are skipped 256
// at a time.
template <int RMAX>
__global__ void __launch_bounds__(kTrdNT) k_trd_backtf_reg(Search* S, TileMap tm) {
  __shared__ double vs[2][32 * RMAX];
  int tile;
  const int si = find_search(tm, tile);
  Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n;
  if (n > 32 * RMAX || trd_bt_blocked(n)) return;  // the blocked form takes these sizes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = tile * trd_bt_cols(n) + warp;
  const bool active = warp < trd_bt_cols(n) && t < n;  // idle warps still join the barriers
  const long long L = s.ldn;
  const double* Vs = s.EA + L * (active ? t : 0);
  double x[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int i = lane + 32 * r;
    x[r] = (active && i < n) ? Vs[i] : 0.0;
  }
  const double* tau = tv(s, TV_TAU);
  const double* Hv = s.EX;
  constexpr int CH = 8;  // registers per chunk: 256 rows
  // stage reflector k - 1 while k is applied
  int cur = 0;
  if (n >= 2) {
    const double* v0 = Hv + L * (n - 2);
    for (int i = threadIdx.x; i < n; i += kTrdNT) vs[0][i] = i > n - 2 ? v0[i] : 0.0;
  }
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    // prefetch the next reflector into registers (stored after this one is applied)
    double pre[(32 * RMAX + kTrdNT - 1) / kTrdNT];
    if (k > 0) {
      const double* vn = Hv + L * (k - 1);
#pragma unroll
      for (int u = 0; u < (32 * RMAX + kTrdNT - 1) / kTrdNT; ++u) {
        const int i = threadIdx.x + kTrdNT * u;
        pre[u] = (i < n && i > k - 1) ? vn[i] : 0.0;
      }
    }
    const double tk = tau[k];
    const double* v = vs[cur];
    if (active && tk != 0.0) {
      double p0 = 0.0, p1 = 0.0;
#pragma unroll
      for (int c = 0; c < RMAX / CH; ++c) {
        if (256 * c + 255 <= k || 256 * c >= n) continue;
#pragma unroll
        for (int rr = 0; rr < CH; rr += 2) {
          const int i0 = lane + 32 * (CH * c + rr), i1 = i0 + 32;
          if (i0 > k && i0 < n) p0 = fma(v[i0], x[CH * c + rr], p0);
          if (i1 > k && i1 < n) p1 = fma(v[i1], x[CH * c + rr + 1], p1);
        }
      }
      const double p = tk * warp_sum_xor(p0 + p1);
#pragma unroll
      for (int c = 0; c < RMAX / CH; ++c) {
        if (256 * c + 255 <= k || 256 * c >= n) continue;
#pragma unroll
        for (int rr = 0; rr < CH; ++rr) {
          const int i = lane + 32 * (CH * c + rr);
          if (i > k && i < n) x[CH * c + rr] = fma(-p, v[i], x[CH * c + rr]);
        }
      }
    }
    if (k > 0) {
#pragma unroll
      for (int u = 0; u < (32 * RMAX + kTrdNT - 1) / kTrdNT; ++u) {
        const int i = threadIdx.x + kTrdNT * u;
        if (i < 32 * RMAX) vs[cur ^ 1][i] = pre[u];
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  if (!active) return;
  // sign: the entry of largest magnitude (the first on ties) positive
  double best = -1.0, val = 0.0;
  int bi = 0x7fffffff;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int i = lane + 32 * r;
    const double a = fabs(x[r]);
    if (i < n && a > best) {
      best = a;
      val = x[r];
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const double ov = __shfl_xor_sync(0xffffffffu, val, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      val = ov;
      bi = oi;
    }
  }
  const double sg = val < 0.0 ? -1.0 : 1.0;
  double* Bc = s.B + L * ti(s, TI_RANK)[t];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int i = lane + 32 * r;
    if (i < n) Bc[i] = sg * x[r];
  }
}

// --------------------------------------------------------------------------
// Eigenvalues with the PD guard (as in the Jacobi route), D, the work counter.
// --------------------------------------------------------------------------
constexpr double kTrdPdFloor = 1e-16;

__global__ void __launch_bounds__(kTrdNT) k_trd_finish(Search* S, int s0) {
  Search& s = S[s0 + blockIdx.x];
  if (!trd_due(s)) return;
  const int n = s.n;
  const long long L = s.ldn;
  const double* lams = tv(s, TV_LAMS);
  const double lo = lams[0], hi = lams[n - 1];
  const double add = (lo < hi * kTrdPdFloor) ? hi * kTrdPdFloor - lo : 0.0;
  for (int i = threadIdx.x; i < n; i += kTrdNT) {
    s.D[i] = sqrt(lams[i] + add);
    if (add != 0.0) s.C[i + L * i] += add;
  }
  if (threadIdx.x == 0) {
    s.eig_sweeps = 0;
    s.eig_count += 1;
  }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
size_t trd_reduce_smem(int max_n, int blocked) { return static_cast<size_t>(max_n) * (blocked ? 8 : 24); }

int trd_reduce_blocks_per_sm(int max_n, int blocked) {
  int b = 0;
  const size_t smem = trd_reduce_smem(max_n, blocked);
  const void* fn = blocked ? reinterpret_cast<const void*>(k_trd_panel) : reinterpret_cast<const void*>(k_trd_sytrd);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kTrdNT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

void trd_set_attributes(int max_n) {
  cudaFuncSetAttribute(k_trd_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(trd_reduce_smem(max_n, 1)));
  cudaFuncSetAttribute(k_trd_sytrd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(trd_reduce_smem(max_n, 0)));
  cudaFuncSetAttribute(k_trd_s2k, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  cudaFuncSetAttribute(k_trd_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  bt_set_attributes();
}

// marks (optional, kTrdStages + 1 events): recorded before the reduction and
// after each stage (reduction, eigenvalues, inverse iteration, Gram-Schmidt in
// clusters, orthogonalisation, back-transformation), for the per-stage times
// of the profiling mode.
int launch_eig_trd(Search* S, const int4* grp, const TrdChunk* chunks, int nchunks, unsigned* bars,
                   int bar_count, int s0, int s1, const TrdMaps& tm, int max_n, int bis_lanes, cudaStream_t st,
                   cudaEvent_t* marks) {
  if (nchunks <= 0 || s1 <= s0) return 0;
  int nl = 0;
  auto mark = [&](int k) {
    if (marks) cudaEventRecord(marks[k], st);
  };
  mark(0);
  int q_prev = -2;  // chunks of the unblocked form carry panel -1
  for (int c = 0; c < nchunks; ++c) {
    const int q = chunks[c].panel;
    if (q != q_prev) {
      if (q_prev >= 0 && q >= 0 && tm.s2kp.total > 0 && tm.s2k.total > 0) {  // the previous panel's trailing update
        k_trd_s2k_pack<<<tm.s2kp.total, kOzNT, 0, st>>>(S, tm.s2kp, q_prev);
        k_trd_s2k<<<tm.s2k.total, kOzNT, kOzSmem, st>>>(S, tm.s2k, q_prev);
        nl += 2;
      }
      // the group barriers and work counters restart per panel
      cudaMemsetAsync(bars, 0, sizeof(unsigned) * bar_count * kTrdBarStride, st);
      q_prev = q;
    }
    if (chunks[c].count <= 0) continue;
    const bool blocked = q >= 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(chunks[c].count);
    cfg.blockDim = dim3(kTrdNT);
    cfg.dynamicSmemBytes = trd_reduce_smem(max_n, blocked ? 1 : 0);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (blocked) cudaLaunchKernelEx(&cfg, k_trd_panel, S, grp + chunks[c].first, q);
    else cudaLaunchKernelEx(&cfg, k_trd_sytrd, S, grp + chunks[c].first);
    ++nl;
  }
  mark(1);
  k_trd_blocks<<<s1 - s0, kTrdNT, 0, st>>>(S, s0);
  if (bis_lanes > 1) k_trd_bisect<kTrdBisLanes><<<tm.tbis.total, kTrdTT, 0, st>>>(S, tm.tbis);
  else k_trd_bisect<1><<<tm.tt.total, kTrdTT, 0, st>>>(S, tm.tt);
  k_trd_rank<<<s1 - s0, kTrdSortNT, 0, st>>>(S, s0);
  mark(2);
  k_trd_invit<<<tm.tt.total, kTrdTT, 0, st>>>(S, tm.tt);
  mark(3);
  k_trd_mgs<<<dim3(s1 - s0, kTrdMgsCtas), kTrdNT, 0, st>>>(S, s0);
  mark(4);
  for (int pass = 0; pass < kTrdNsSteps; ++pass) {
    if (tm.ozp.total > 0) k_trd_oz_pack<<<tm.ozp.total, kOzNT, 0, st>>>(S, tm.ozp, pass);
    if (tm.ozg.total > 0) k_trd_oz_gram<<<tm.ozg.total, kOzNT, kOzSmem, st>>>(S, tm.ozg, pass);
    k_trd_ns<<<tm.tsq.total, kGNT, 0, st>>>(S, tm.tsq, pass);
  }
  mark(5);
  if (tm.tbt.total > 0) {  // n < kBtBlockedMinN
    k_trd_backtf_reg<16><<<tm.tbt.total, kTrdNT, 0, st>>>(S, tm.tbt);
    ++nl;
  }
  nl += launch_bt(S, tm, max_n, st);  // the larger ones
  k_trd_finish<<<s1 - s0, kTrdNT, 0, st>>>(S, s0);
  mark(6);
  return nl + 6 + 3 * kTrdNsSteps;
}

}  // namespace cmaes_gb300
