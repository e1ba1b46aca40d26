// kernels_jacobi_cluster.cu -- the warm-started parallel Jacobi of
// kernels_eig.cu spread over a thread-block cluster of 8 CTAs per search.
//
// Same method, same rotations, same convergence test and the same canonical
// output as the single-CTA variant; only the data placement differs:
//   * Tournament slots. Pair i of a round-robin step is (T[i], Bt[i]); CTA c
//     owns slots [c spc, (c+1) spc) and keeps the full columns of A and of the
//     eigenvector accumulator V for the players sitting in its slots.
//   * Each step: every CTA computes the rotations of its own pairs (all data
//     local), publishes them, and after a cluster barrier reads everybody's
//     rotations through distributed shared memory. A <- A J (column mixing)
//     and V <- V J touch only the owner's two columns; A <- J^T A (row mixing)
//     touches rows p_i, q_i of every column, so each CTA applies all
//     rotations to its own columns. The 2 x 2 diagonal block of every rotated
//     pair is then set exactly (a_pq = 0, a_pp -= t a_pq, a_qq += t a_pq).
//   * Between steps the players move one place along the ring
//     T[1] -> ... -> T[P-1] -> Bt[P-1] -> ... -> Bt[0] -> T[1] (T[0] fixed),
//     which is the circle method: every pair meets once per N - 1 steps. Moves
//     inside a CTA only relabel buffers; a move across CTAs copies the column
//     (A and V parts) into a landing buffer of the neighbour, followed by a
//     second cluster barrier.
// Control flow is uniform over the cluster: every CTA reads the same search
// flags and the same gathered rotations, so all reach the same barriers.
#include <cmath>
#include <cooperative_groups.h>
#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace cmaes_gb300 {

constexpr int kCS = 8;            // CTAs per cluster (portable size)
constexpr int kCNT = 256;         // threads per CTA
constexpr int kClusterMaxN = 256;
constexpr double kCTol = 1e-14;   // same relative threshold as the single-CTA variant
constexpr int kCMaxSweeps = 40;
constexpr double kCPdFloor = 1e-16;

namespace {

struct CLayout {
  int stride, nbuf, spc, P, N;
  size_t bytes;
  // double arrays
  size_t colA, colV, ac, as, lc, ls, lt, lapp, laqq, lapq, evall;
  // int arrays
  size_t ids, tb, bb, ap, aq, aa, lp, lq, la, nmap;
};

__host__ __device__ inline CLayout make_layout(int max_n) {
  CLayout L;
  L.N = max_n + (max_n & 1);
  L.P = L.N / 2;
  L.spc = (L.P + kCS - 1) / kCS;
  L.nbuf = 2 * L.spc + 2;
  L.stride = max_n + 1;
  size_t d = 0;
  L.colA = d; d += static_cast<size_t>(L.nbuf) * L.stride;
  L.colV = d; d += static_cast<size_t>(L.nbuf) * L.stride;
  L.ac = d; d += L.P;
  L.as = d; d += L.P;
  L.lc = d; d += L.spc;
  L.ls = d; d += L.spc;
  L.lt = d; d += L.spc;
  L.lapp = d; d += L.spc;
  L.laqq = d; d += L.spc;
  L.lapq = d; d += L.spc;
  L.evall = d; d += L.N;
  size_t i = 0;
  L.ids = i; i += L.nbuf;
  L.tb = i; i += L.spc;
  L.bb = i; i += L.spc;
  L.ap = i; i += L.P;
  L.aq = i; i += L.P;
  L.aa = i; i += L.P;
  L.lp = i; i += L.spc;
  L.lq = i; i += L.spc;
  L.la = i; i += L.spc;
  L.nmap = i; i += 2 * L.spc + 8;  // new slot map and copy plan
  L.bytes = d * 8 + i * 4 + 16;
  return L;
}

}  // namespace

size_t jacobi_cluster_smem_bytes(int max_n) { return make_layout(max_n).bytes; }
int jacobi_cluster_max_n() { return kClusterMaxN; }

__global__ void __cluster_dims__(kCS, 1, 1) __launch_bounds__(kCNT)
    k_jacobi_cluster(Search* S, int s0, int lo_n, int hi_n, int layout_n) {
  extern __shared__ double dsm[];
  __shared__ double shr[32];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = static_cast<int>(cl.block_rank());
  Search& s = S[s0 + static_cast<int>(blockIdx.x) / kCS];
  // uniform over the cluster: every CTA reads the same flags
  if (s.done || !s.eig_due || s.n <= lo_n || s.n > hi_n) return;

  const CLayout L = make_layout(layout_n);
  double* colA = dsm + L.colA;
  double* colV = dsm + L.colV;
  double* ac = dsm + L.ac;
  double* as = dsm + L.as;
  double* lc = dsm + L.lc;
  double* ls = dsm + L.ls;
  double* lt = dsm + L.lt;
  double* lapp = dsm + L.lapp;
  double* laqq = dsm + L.laqq;
  double* lapq = dsm + L.lapq;
  double* evall = dsm + L.evall;
  int* ibase = reinterpret_cast<int*>(dsm + (L.evall + L.N));
  int* ids = ibase + L.ids;
  int* tb = ibase + L.tb;
  int* bb = ibase + L.bb;
  int* ap = ibase + L.ap;
  int* aq = ibase + L.aq;
  int* aa = ibase + L.aa;
  int* lp = ibase + L.lp;
  int* lq = ibase + L.lq;
  int* la = ibase + L.la;
  int* nmap = ibase + L.nmap;  // [0, spc): new tb, [spc, 2spc): new bb, then copy plan

  const int n = s.n, ldn = s.ldn;
  const int N = n + (n & 1), P = N / 2;
  const int spc = (P + kCS - 1) / kCS;
  const int g0 = min(P, crank * spc), g1 = min(P, g0 + spc), nloc = g1 - g0;
  const int st = L.stride;
  const int IN_TOP = 2 * spc, IN_BOT = 2 * spc + 1;
  const int tid = threadIdx.x;

  // initial seating T[i] = 2i, Bt[i] = 2i + 1; buffer b of this CTA holds
  // player 2 g0 + b; A symmetrised from EA = B^T C B, V = B
  for (int k = tid; k < nloc; k += kCNT) {
    tb[k] = 2 * k;
    bb[k] = 2 * k + 1;
  }
  for (int b = tid; b < 2 * nloc; b += kCNT) ids[b] = 2 * g0 + b;
  for (int e = tid; e < 2 * nloc * n; e += kCNT) {
    const int b = e / n, r = e % n, id = 2 * g0 + b;
    double a = 0.0, v = 0.0;
    if (id < n) {
      a = 0.5 * (s.EA[r + static_cast<long long>(ldn) * id] + s.EA[id + static_cast<long long>(ldn) * r]);
      v = s.B[r + static_cast<long long>(ldn) * id];
    }
    colA[b * st + r] = a;
    colV[b * st + r] = v;
  }
  __syncthreads();

  long long rotations = 0;
  int sweeps = 0;
  // every pair meets once in any N - 1 consecutive steps, so N - 1 steps in a
  // row without a rotation mean convergence (same result as a quiet sweep)
  int quiet = 0;
  bool converged = false;
  for (; sweeps < kCMaxSweeps && !converged; ++sweeps) {
    for (int step = 0; step < N - 1; ++step) {
      // (1) rotations of the local pairs
      for (int k = tid; k < nloc; k += kCNT) {
        const int bp = tb[k], bq = bb[k];
        const int p = ids[bp], q = ids[bq];
        double c = 1.0, sn = 0.0, tn = 0.0, app = 0.0, aqq = 0.0, apq = 0.0;
        int act = 0;
        if (p < n && q < n) {
          app = colA[bp * st + p];
          aqq = colA[bq * st + q];
          apq = colA[bq * st + p];
          if (apq != 0.0 && fabs(apq) > kCTol * sqrt(fabs(app * aqq))) {
            const double theta = (aqq - app) / (2.0 * apq);
            const double at = fabs(theta);
            tn = (at > 1e150) ? 0.5 / theta : (theta >= 0.0 ? 1.0 : -1.0) / (at + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(tn * tn + 1.0);
            sn = tn * c;
            act = 1;
          }
        }
        lc[k] = c;
        ls[k] = sn;
        lt[k] = tn;
        lapp[k] = app;
        laqq[k] = aqq;
        lapq[k] = apq;
        lp[k] = p;
        lq[k] = q;
        la[k] = act;
      }
      cl.sync();  // rotations published
      // (2) gather every pair's rotation
      int any = 0;
      for (int i = tid; i < P; i += kCNT) {
        const int owner = i / spc, k = i - owner * spc;
        const double* rc = cl.map_shared_rank(lc, owner);
        const double* rs = cl.map_shared_rank(ls, owner);
        const int* rp = cl.map_shared_rank(lp, owner);
        const int* rq = cl.map_shared_rank(lq, owner);
        const int* ra = cl.map_shared_rank(la, owner);
        ac[i] = rc[k];
        as[i] = rs[k];
        ap[i] = rp[k];
        aq[i] = rq[k];
        aa[i] = ra[k];
        any |= ra[k];
      }
      any = __syncthreads_or(any);
      quiet = any ? 0 : quiet + 1;
      if (quiet >= N - 1) {
        converged = true;
        break;  // uniform: every CTA gathered the same rotations
      }
      if (any) {
        // (3) A <- A J and V <- V J on the local pairs' columns
        for (int e = tid; e < nloc * n; e += kCNT) {
          const int k = e / n, r = e % n;
          if (!la[k]) continue;
          const double c = lc[k], sn = ls[k];
          double* Ap = colA + tb[k] * st;
          double* Aq = colA + bb[k] * st;
          const double x = Ap[r], y = Aq[r];
          Ap[r] = c * x - sn * y;
          Aq[r] = sn * x + c * y;
          double* Vp = colV + tb[k] * st;
          double* Vq = colV + bb[k] * st;
          const double v = Vp[r], w = Vq[r];
          Vp[r] = c * v - sn * w;
          Vq[r] = sn * v + c * w;
        }
        __syncthreads();
        // (4) A <- J^T A: rows p_i, q_i of every local column
        for (int e = tid; e < 2 * nloc * P; e += kCNT) {
          const int lb = e / P, i = e - lb * P;
          if (!aa[i]) continue;
          const int buf = lb < nloc ? tb[lb] : bb[lb - nloc];
          double* col = colA + buf * st;
          const int p = ap[i], q = aq[i];
          const double c = ac[i], sn = as[i];
          const double x = col[p], y = col[q];
          col[p] = c * x - sn * y;
          col[q] = sn * x + c * y;
        }
        __syncthreads();
        // (5) exact 2 x 2 diagonal block of each rotated local pair
        for (int k = tid; k < nloc; k += kCNT) {
          if (!la[k]) continue;
          const int p = lp[k], q = lq[k];
          double* Ap = colA + tb[k] * st;
          double* Aq = colA + bb[k] * st;
          Ap[p] = lapp[k] - lt[k] * lapq[k];
          Aq[q] = laqq[k] + lt[k] * lapq[k];
          Ap[q] = 0.0;
          Aq[p] = 0.0;
        }
        if (tid == 0) {
          int cnt = 0;
          for (int i = 0; i < P; ++i) cnt += aa[i];
          rotations += cnt;
        }
        __syncthreads();
      }
      // (6) ring move: send the leaving columns to the neighbours' landing buffers
      // top side: T[g1-1] -> T[g1] of CTA c+1 (T[0] never moves; T[P-1] stays local)
      // bottom side: Bt[g0] -> Bt[g0-1] of CTA c-1; Bt[0] -> T[1] (CTA 1 when spc == 1)
      int send_top = -1, send_bot = -1, dst_bot = -1, land_bot = -1;
      if (nloc > 0) {
        if (g1 < P && g1 - 1 > 0) send_top = tb[nloc - 1];
        if (g0 >= 1) { send_bot = bb[0]; dst_bot = crank - 1; land_bot = IN_BOT; }
        else if (nloc == 1 && P > 1) { send_bot = bb[0]; dst_bot = crank + 1; land_bot = IN_TOP; }
      }
      if (send_top >= 0) {
        double* rA = cl.map_shared_rank(colA, crank + 1) + IN_TOP * st;
        double* rV = cl.map_shared_rank(colV, crank + 1) + IN_TOP * st;
        for (int r = tid; r < n; r += kCNT) {
          rA[r] = colA[send_top * st + r];
          rV[r] = colV[send_top * st + r];
        }
        if (tid == 0) cl.map_shared_rank(ids, crank + 1)[IN_TOP] = ids[send_top];
      }
      if (send_bot >= 0) {
        double* rA = cl.map_shared_rank(colA, dst_bot) + land_bot * st;
        double* rV = cl.map_shared_rank(colV, dst_bot) + land_bot * st;
        for (int r = tid; r < n; r += kCNT) {
          rA[r] = colA[send_bot * st + r];
          rV[r] = colV[send_bot * st + r];
        }
        if (tid == 0) cl.map_shared_rank(ids, dst_bot)[land_bot] = ids[send_bot];
      }
      cl.sync();  // columns delivered
      // (7) relabel: new seating of the local slots, landing buffers copied
      // into the buffers that were sent away
      if (tid == 0 && nloc > 0) {
        int* ntb = nmap;
        int* nbb = nmap + spc;
        int* plan = nmap + 2 * spc;  // (landing, target) pairs, up to two
        int np = 0;
        int freed[2], nf = 0;
        if (send_top >= 0) freed[nf++] = send_top;
        if (send_bot >= 0) freed[nf++] = send_bot;
        for (int k = nloc - 1; k >= 1; --k) ntb[k] = tb[k - 1];
        if (g0 == 0) {
          ntb[0] = tb[0];
          if (nloc >= 2) ntb[1] = bb[0];
        } else {
          const int f = freed[--nf];
          plan[2 * np] = IN_TOP;
          plan[2 * np + 1] = f;
          ++np;
          ntb[0] = f;
        }
        for (int k = 0; k < nloc - 1; ++k) nbb[k] = bb[k + 1];
        if (g1 == P) {
          nbb[nloc - 1] = tb[nloc - 1];
        } else {
          const int f = freed[--nf];
          plan[2 * np] = IN_BOT;
          plan[2 * np + 1] = f;
          ++np;
          nbb[nloc - 1] = f;
        }
        for (int k = 0; k < nloc; ++k) {
          tb[k] = ntb[k];
          bb[k] = nbb[k];
        }
        plan[4] = np;
      }
      __syncthreads();
      if (nloc > 0) {
        const int* plan = nmap + 2 * spc;
        const int np = plan[4];
        for (int e = tid; e < np * n; e += kCNT) {
          const int j = e / n, r = e % n;
          const int from = plan[2 * j], to = plan[2 * j + 1];
          colA[to * st + r] = colA[from * st + r];
          colV[to * st + r] = colV[from * st + r];
        }
        if (tid < np) ids[plan[2 * tid + 1]] = ids[plan[2 * tid]];
      }
      __syncthreads();
    }
  }

  // eigenvalues into every CTA's evall
  for (int lb = tid; lb < 2 * nloc; lb += kCNT) {
    const int buf = lb < nloc ? tb[lb] : bb[lb - nloc];
    const int id = ids[buf];
    if (id >= n) continue;
    const double ev = colA[buf * st + id];
    for (int c = 0; c < kCS; ++c) cl.map_shared_rank(evall, c)[id] = ev;
  }
  cl.sync();
  double lo = INFINITY, hi = -INFINITY;
  for (int i = tid; i < n; i += kCNT) {
    lo = fmin(lo, evall[i]);
    hi = fmax(hi, evall[i]);
  }
  hi = block_max<kCNT>(hi, shr);
  lo = -block_max<kCNT>(-lo, shr);
  const double add = (lo < hi * kCPdFloor) ? hi * kCPdFloor - lo : 0.0;
  // canonical representative: ascending eigenvalue (ties by index), largest
  // entry of each column positive; one warp per local column
  const int lane = tid & 31, warp = tid >> 5;
  for (int lb = warp; lb < 2 * nloc; lb += kCNT / 32) {
    const int buf = lb < nloc ? tb[lb] : bb[lb - nloc];
    const int id = ids[buf];
    if (id >= n) continue;
    const double e = evall[id];
    int r = 0;
    for (int j = lane; j < n; j += 32) r += (evall[j] < e) || (evall[j] == e && j < id);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    const double* v = colV + buf * st;
    double best = -1.0, val = 0.0;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      const double a = fabs(v[i]);
      if (a > best) { best = a; val = v[i]; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const double ov = __shfl_xor_sync(0xffffffffu, val, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; val = ov; bi = oi; }
    }
    const double sg = (val < 0.0) ? -1.0 : 1.0;
    double* dst = s.B + static_cast<long long>(ldn) * r;
    for (int i = lane; i < n; i += 32) dst[i] = sg * v[i];
    if (lane == 0) s.D[r] = sqrt(e + add);
  }
  if (crank == 0) {
    if (add != 0.0)
      for (int i = tid; i < n; i += kCNT) s.C[i + static_cast<long long>(ldn) * i] += add;
    if (tid == 0) {
      const int done_sweeps = sweeps;
      s.eig_sweeps = done_sweeps;
      s.eig_count += 1;
      s.eig_sweeps_total += done_sweeps;
      s.eig_rotations += rotations;
    }
  }
  cl.sync();  // no CTA leaves while another may still touch its shared memory
}

void launch_jacobi_cluster(Search* S, int s0, int s1, int lo_n, int hi_n, int layout_n, cudaStream_t st) {
  if (s1 <= s0 || layout_n <= lo_n) return;
  const size_t bytes = jacobi_cluster_smem_bytes(layout_n);
  cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  k_jacobi_cluster<<<(s1 - s0) * kCS, kCNT, bytes, st>>>(S, s0, lo_n, hi_n, layout_n);
}

}  // namespace cmaes_gb300
