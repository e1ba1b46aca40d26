// kernels_jacobi_cluster.cu -- the warm-started parallel Jacobi of
// kernels_eig.cu spread over a thread-block cluster of 8 CTAs per search.
//
// Same method, same rotations, same convergence test and the same canonical
// output as the single-CTA variant; only the data placement differs:
//   * Tournament slots. Pair i of a round-robin step is (T[i], Bt[i]); CTA c
//     owns slots [c spc, (c+1) spc) and keeps the full columns of A and of the
//     eigenvector accumulator V for the players sitting in its slots. One warp
//     serves one slot.
//   * Each step: lane j of warp 0 computes the rotation of local slot j from
//     the slot's two columns (one lane per pair keeps the FP64 work of the
//     rotations to one warp instruction stream per CTA) and writes it into the
//     rotation table of every CTA of the cluster (distributed shared memory);
//     p, q and the rotate flag travel packed in one word. After a cluster
//     barrier each warp
//     applies A <- A J and V <- V J to its two columns (column mixing), then
//     A <- J^T A to the rows p_i, q_i of its two columns for every rotated pair
//     (row mixing), then sets its pair's 2 x 2 diagonal block exactly
//     (a_pq = 0, a_pp - t a_pq, a_qq + t a_pq). All of this is warp-local.
//   * Between steps the players move one place along the ring
//     T[1] -> ... -> T[P-1] -> Bt[P-1] -> ... -> Bt[0] -> T[1] (T[0] fixed),
//     the circle method: every pair meets once in any N - 1 steps. A column
//     leaving the CTA is written into a landing buffer of the neighbour; a
//     second cluster barrier separates those writes from their use.
// The two cluster barriers are the only synchronisation of a step. Control
// flow is uniform over the cluster: every CTA reads the same search flags and
// the same rotation table, so all reach the same barriers.
#include <cmath>
#include <cooperative_groups.h>
#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace cmaes_gb300 {

constexpr int kCS = 8;            // CTAs per cluster (portable size)
constexpr int kClusterMaxN = 256;
constexpr double kCTol = 1e-14;   // same relative threshold as the single-CTA variant
constexpr int kCMaxSweeps = 40;
constexpr double kCPdFloor = 1e-16;

namespace {

struct CLayout {
  int stride, nbuf, spc, P, N, threads;
  size_t bytes;
  size_t colA, colV, rc, rs, rt, evall;  // double arrays
  size_t ids, rpq, map;                  // int arrays
};

__host__ __device__ inline CLayout make_layout(int max_n) {
  CLayout L;
  L.N = max_n + (max_n & 1);
  L.P = L.N / 2;
  L.spc = (L.P + kCS - 1) / kCS;
  L.nbuf = 2 * L.spc + 2;
  L.stride = max_n + 1;
  L.threads = 32 * (L.spc > 2 ? L.spc : 2);
  size_t d = 0;
  L.colA = d; d += static_cast<size_t>(L.nbuf) * L.stride;
  L.colV = d; d += static_cast<size_t>(L.nbuf) * L.stride;
  L.rc = d; d += L.P;
  L.rs = d; d += L.P;
  L.rt = d; d += L.P;
  L.evall = d; d += L.N;
  size_t i = 0;
  L.ids = i; i += L.nbuf;
  L.rpq = i; i += L.P;
  L.map = i; i += 4 * L.spc;  // two parities x (top, bottom) buffer of each local slot
  L.bytes = d * 8 + i * 4 + 16;
  return L;
}

}  // namespace

size_t jacobi_cluster_smem_bytes(int max_n) { return make_layout(max_n).bytes; }
int jacobi_cluster_max_n() { return kClusterMaxN; }

__global__ void __cluster_dims__(kCS, 1, 1) __launch_bounds__(512)
    k_jacobi_cluster(Search* S, int s0, int lo_n, int hi_n, int layout_n) {
  extern __shared__ double dsm[];
  __shared__ double shr[32];
  __shared__ int shf[kCS];  // convergence verdict of each CTA of the cluster
  __shared__ double shm[kCS];  // max |a_ii| over each CTA's columns
  cg::cluster_group cl = cg::this_cluster();
  const int crank = static_cast<int>(cl.block_rank());
  Search& s = S[s0 + static_cast<int>(blockIdx.x) / kCS];
  // uniform over the cluster: every CTA reads the same flags
  if (s.done || !s.eig_due || s.trd || s.n <= lo_n || s.n > hi_n) return;

  const CLayout L = make_layout(layout_n);
  double* colA = dsm + L.colA;
  double* colV = dsm + L.colV;
  double* rc = dsm + L.rc;
  double* rs = dsm + L.rs;
  double* rt = dsm + L.rt;
  double* evall = dsm + L.evall;
  int* ibase = reinterpret_cast<int*>(dsm + (L.evall + L.N));
  int* ids = ibase + L.ids;
  int* rpq = ibase + L.rpq;  // p | q << 12 | rotate << 24 (n <= 256)
  int* map = ibase + L.map;  // map[par * 2 spc + 2 k] = top buffer, +1 = bottom buffer

  const int n = s.n, ldn = s.ldn;
  const int N = n + (n & 1), P = N / 2;
  const int spc = (P + kCS - 1) / kCS;
  const int g0 = min(P, crank * spc), g1 = min(P, g0 + spc), nloc = g1 - g0;
  const int st = L.stride;
  const int IN_TOP = 2 * spc, IN_BOT = 2 * spc + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool mine = warp < nloc;  // this warp serves local slot `warp`
  const int k = warp;

  // initial seating T[i] = 2i, Bt[i] = 2i + 1: buffer b of this CTA holds
  // player 2 g0 + b; A symmetrised from EA = B^T C B, V = B
  for (int b = tid; b < 2 * nloc; b += blockDim.x) ids[b] = 2 * g0 + b;
  for (int i = tid; i < nloc; i += blockDim.x) {
    map[2 * i] = 2 * i;
    map[2 * i + 1] = 2 * i + 1;
  }
  for (int e = tid; e < 2 * nloc * n; e += blockDim.x) {
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
  // On the refined route A = X^T C X comes from FP64 products whose rounding
  // reaches n eps64 max|a_ii| (the bound for a length-n dot product of the
  // unit columns of X with those of C X); entries below that are noise and
  // are not rotated: one such bound on FP64 handles (a rotation it skips moves
  // an eigenvector by at most n eps64 / relative gap), four on mixed-precision
  // handles, whose contract is a backward error of 1e-12. Elsewhere floor = 0:
  // the plain relative test.
  double floor_abs = 0.0;
  if (eig_refined_route(s)) {
    if (warp == 0) {
      double m = 0.0;
      for (int b = lane; b < 2 * nloc; b += 32) {
        const int id = 2 * g0 + b;
        if (id < n) m = fmax(m, fabs(colA[b * st + id]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane < kCS) cl.map_shared_rank(shm, lane)[crank] = m;
    }
    cl.sync();
    double amax = 0.0;
#pragma unroll
    for (int c = 0; c < kCS; ++c) amax = fmax(amax, shm[c]);
    floor_abs = (s.mixed ? 4.0 : 1.0) * n * 0x1p-53 * amax;
  }

  long long rotations = 0;
  int sweeps = 0, quiet = 0, par = 0;
  bool converged = false;
  for (; sweeps < kCMaxSweeps && !converged; ++sweeps) {
    for (int step = 0; step < N - 1; ++step) {
      const int* mp = map + par * 2 * spc;
      if (warp == 0 && lane < nloc) {  // rotation of local slot `lane`
        const int ft = mp[2 * lane], fb = mp[2 * lane + 1];
        const int p = ids[ft], q = ids[fb];
        double c = 1.0, sn = 0.0, tn = 0.0;
        int act = 0;
        if (p < n && q < n) {
          const double app = colA[ft * st + p], aqq = colA[fb * st + q], apq = colA[fb * st + p];
          if (jacobi_rotates(app, aqq, apq, kCTol * kCTol, floor_abs)) {
            jacobi_rotation(app, aqq, apq, tn, c, sn);
            act = 1;
          }
        }
        const int gi = g0 + lane;
        const int pq = p | (q << 12) | (act << 24);
        rt[gi] = tn;
#pragma unroll
        for (int cc = 0; cc < kCS; ++cc) {
          cl.map_shared_rank(rc, cc)[gi] = c;
          cl.map_shared_rank(rs, cc)[gi] = sn;
          cl.map_shared_rank(rpq, cc)[gi] = pq;
        }
      }
      cl.sync();  // rotation table complete everywhere
      int cnt = 0;
      for (int i = lane; i < P; i += 32) cnt += rpq[i] >> 24;
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (tid == 0 && crank == 0) rotations += cnt;
      if (cnt) {
        quiet = 0;
      } else if (++quiet == 1 || (quiet & 15) == 0) {
        // a quiet step: if no off-diagonal entry passes the test any more, the
        // rest of the quiet window would change nothing. Diagonal entries go to
        // every CTA, each warp tests the upper part of its two columns, and the
        // verdicts meet in every CTA's flag slots.
        if (mine && lane < kCS) {
          const int ft = mp[2 * k], fb = mp[2 * k + 1];
          const int p = ids[ft], q = ids[fb];
          double* ev = cl.map_shared_rank(evall, lane);
          if (p < n) ev[p] = colA[ft * st + p];
          if (q < n) ev[q] = colA[fb * st + q];
        }
        cl.sync();
        int pend = 0;
        if (mine) {
          for (int h = 0; h < 2; ++h) {
            const int buf = mp[2 * k + h];
            const int id = ids[buf];
            if (id >= n) continue;
            const double ajj = evall[id];
            const double* col = colA + buf * st;
            for (int r = lane; r < id; r += 32)
              pend |= jacobi_rotates(evall[r], ajj, col[r], kCTol * kCTol, floor_abs);
          }
        }
        pend = __syncthreads_or(pend);
        if (tid < kCS) cl.map_shared_rank(shf, tid)[crank] = pend;
        cl.sync();
        int open = 0;
#pragma unroll
        for (int c = 0; c < kCS; ++c) open |= shf[c];
        if (!open) quiet = N - 1;
      }
      if (quiet >= N - 1) {
        converged = true;
        break;  // uniform: every warp of the cluster saw the same table and flags
      }
      int bt = 0, bb = 0;
      if (mine) {
        bt = mp[2 * k];
        bb = mp[2 * k + 1];
      }
      if (mine && cnt) {
        const int gi = g0 + k;
        const int pq = rpq[gi];
        const int act = pq >> 24, p = pq & 0xfff, q = (pq >> 12) & 0xfff;
        double* At = colA + bt * st;
        double* Ab = colA + bb * st;
        double app = 0.0, aqq = 0.0, apq = 0.0;
        if (act) {  // A <- A J and V <- V J on the pair's columns
          app = At[p];
          aqq = Ab[q];
          apq = Ab[p];
          const double c = rc[gi], sn = rs[gi];
          double* Vt = colV + bt * st;
          double* Vb = colV + bb * st;
          __syncwarp();  // the block entries are read before any lane overwrites them
          for (int r = lane; r < n; r += 32) {
            const double x = At[r], y = Ab[r];
            At[r] = c * x - sn * y;
            Ab[r] = sn * x + c * y;
            const double v = Vt[r], w = Vb[r];
            Vt[r] = c * v - sn * w;
            Vb[r] = sn * v + c * w;
          }
          __syncwarp();
        }
        // A <- J^T A: rows p_i, q_i of both columns, every rotated pair
        for (int i = lane; i < P; i += 32) {
          const int pqi = rpq[i];
          if (!(pqi >> 24)) continue;
          const int pi = pqi & 0xfff, qi = (pqi >> 12) & 0xfff;
          const double ci = rc[i], si = rs[i];
          double x = At[pi], y = At[qi];
          At[pi] = ci * x - si * y;
          At[qi] = si * x + ci * y;
          x = Ab[pi];
          y = Ab[qi];
          Ab[pi] = ci * x - si * y;
          Ab[qi] = si * x + ci * y;
        }
        __syncwarp();
        if (act && lane == 0) {  // exact 2 x 2 diagonal block
          const double tn = rt[gi];
          At[p] = app - tn * apq;
          Ab[q] = aqq + tn * apq;
          At[q] = 0.0;
          Ab[p] = 0.0;
        }
        __syncwarp();
      }
      // ring move: the top column of the last local slot goes to CTA c+1
      // (T[0] never moves, T[P-1] stays local as Bt[P-1]); the bottom column of
      // the first local slot goes to CTA c-1 (Bt[0] -> T[1], at CTA 1 when
      // spc == 1)
      if (mine && k == nloc - 1 && g1 < P && g1 - 1 > 0) {
        double* rA = cl.map_shared_rank(colA, crank + 1) + IN_TOP * st;
        double* rV = cl.map_shared_rank(colV, crank + 1) + IN_TOP * st;
        for (int r = lane; r < n; r += 32) {
          rA[r] = colA[bt * st + r];
          rV[r] = colV[bt * st + r];
        }
        if (lane == 0) cl.map_shared_rank(ids, crank + 1)[IN_TOP] = ids[bt];
      }
      if (mine && k == 0 && (g0 >= 1 || (nloc == 1 && P > 1))) {
        const int dst = g0 >= 1 ? crank - 1 : crank + 1;
        const int land = g0 >= 1 ? IN_BOT : IN_TOP;
        double* rA = cl.map_shared_rank(colA, dst) + land * st;
        double* rV = cl.map_shared_rank(colV, dst) + land * st;
        for (int r = lane; r < n; r += 32) {
          rA[r] = colA[bb * st + r];
          rV[r] = colV[bb * st + r];
        }
        if (lane == 0) cl.map_shared_rank(ids, dst)[land] = ids[bb];
      }
      cl.sync();  // columns delivered
      // new seating of this warp's slot (computed from the old map, written
      // to the other parity); landing buffers are copied by the warp that
      // takes them over
      if (mine) {
        int* nm = map + (par ^ 1) * 2 * spc;
        int ntop, nbot, copy_top = 0, copy_bot = 0;
        if (k >= 1) ntop = (g0 == 0 && k == 1) ? mp[1] : mp[2 * (k - 1)];
        else if (g0 == 0) ntop = mp[0];
        else { ntop = mp[1]; copy_top = 1; }  // old Bt[g0] buffer takes the incoming T[g0]
        if (k < nloc - 1) nbot = mp[2 * (k + 1) + 1];
        else if (g1 == P) nbot = mp[2 * (nloc - 1)];
        else {
          nbot = (g0 == 0 && nloc == 1) ? mp[1] : mp[2 * (nloc - 1)];
          copy_bot = 1;
        }
        if (copy_top) {
          for (int r = lane; r < n; r += 32) {
            colA[ntop * st + r] = colA[IN_TOP * st + r];
            colV[ntop * st + r] = colV[IN_TOP * st + r];
          }
          if (lane == 0) ids[ntop] = ids[IN_TOP];
        }
        if (copy_bot) {
          for (int r = lane; r < n; r += 32) {
            colA[nbot * st + r] = colA[IN_BOT * st + r];
            colV[nbot * st + r] = colV[IN_BOT * st + r];
          }
          if (lane == 0) ids[nbot] = ids[IN_BOT];
        }
        if (lane == 0) {
          nm[2 * k] = ntop;
          nm[2 * k + 1] = nbot;
        }
        __syncwarp();
      }
      par ^= 1;
      __syncthreads();  // new seating visible to every warp
    }
  }

  // eigenvalues into every CTA's evall
  const int* mp = map + par * 2 * spc;
  for (int lb = tid; lb < 2 * nloc; lb += blockDim.x) {
    const int buf = mp[lb];
    const int id = ids[buf];
    if (id >= n) continue;
    const double ev = colA[buf * st + id];
    for (int cc = 0; cc < kCS; ++cc) cl.map_shared_rank(evall, cc)[id] = ev;
  }
  cl.sync();
  double lo = INFINITY, hi = -INFINITY;
  for (int i = tid; i < n; i += blockDim.x) {
    lo = fmin(lo, evall[i]);
    hi = fmax(hi, evall[i]);
  }
  // block_max expects 512 threads worth of warps; blockDim is a multiple of 32
  {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    }
    if (lane == 0) {
      shr[warp] = hi;
      shr[16 + warp] = lo;
    }
    __syncthreads();
    hi = -INFINITY;
    lo = INFINITY;
    for (int w = 0; w < static_cast<int>(blockDim.x) / 32; ++w) {
      hi = fmax(hi, shr[w]);
      lo = fmin(lo, shr[16 + w]);
    }
  }
  const double add = (lo < hi * kCPdFloor) ? hi * kCPdFloor - lo : 0.0;
  // canonical representative: ascending eigenvalue (ties by index), largest
  // entry of each column positive; one warp per local column
  for (int lb = warp; lb < 2 * nloc; lb += blockDim.x / 32) {
    const int buf = mp[lb];
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
      for (int i = tid; i < n; i += blockDim.x) s.C[i + static_cast<long long>(ldn) * i] += add;
    if (tid == 0) {
      s.eig_sweeps = sweeps;
      s.eig_count += 1;
      s.eig_sweeps_total += sweeps;
      s.eig_rotations += rotations;
    }
  }
  cl.sync();  // no CTA leaves while another may still touch its shared memory
}

void launch_jacobi_cluster(Search* S, int s0, int s1, int lo_n, int hi_n, int layout_n, cudaStream_t st) {
  if (s1 <= s0 || layout_n <= lo_n) return;
  const CLayout L = make_layout(layout_n);
  cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L.bytes));
  k_jacobi_cluster<<<(s1 - s0) * kCS, L.threads, L.bytes, st>>>(S, s0, lo_n, hi_n, layout_n);
}

}  // namespace cmaes_gb300
