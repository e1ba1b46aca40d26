// kernels_eig_big.cu -- the FP32 Jacobi stage of the refined eigensolver route
// for n > kEigMixedMaxN, where A32 no longer fits one CTA's shared memory.
//
// The arithmetic is that of k_jacobi32 (kernels_eig_mixed.cu): A32 = 2^-k
// (B^T C B - c I), round-robin cyclic Jacobi with the matrix moving with the
// ring, rotations below FP32 resolution skipped, rotations logged and V32
// formed afterwards by replaying the log on the rows of I. Here a step is one
// kernel launch over all large searches of the batch: every thread owns one
// off-diagonal 2 x 2 block, reads it from one buffer in global memory (L2),
// rotates it and writes its four entries to their positions of the next step
// in the other buffer; the threads owning the P role blocks form the next
// step's rotations. The kernel boundary is the step's barrier: no block ever
// waits for another.
//
// Buffer layout (floats, NB = P (P - 1) / 2 off-diagonal blocks): planes
// 2x + y at pl NB + slot(K, L) for the entry between ring positions (K, x)
// and (L, y), K < L; then a_aa, a_ab, a_bb of the diagonal blocks at
// 4 NB + {0, P, 2P} + K. Slots follow the thread list, diagonal by diagonal
// d = L - K: the P role blocks first ((0, 1), (0, 2), (k - 1, k + 1),
// (P - 2, P - 1) for next-step pair k), then d = 1 (K = 1 .. P - 3), then
// d = 3, 4, ..., P - 1 (K = 0 .. P - 1 - d). The ring turn moves an entry
// along its diagonal or two diagonals over, so consecutive threads read and
// write (mostly) consecutive words.
//
// Convergence: the role threads record the last step that rotates anything
// (atomicMax); a step N - 1 steps after it would only turn the ring, so every
// later launch returns at once (the full quiet window of the cyclic method).
// Every 64 steps a check over the whole matrix ends the window early: if the
// coming step rotates nothing and no entry passes the test, nothing ever will
// (the last CTA of the check decides, after a threadfence; no CTA waits).
// The host checks the searches once per sweep of the largest one and stops
// launching when all have converged or spent kJ32BigSweeps sweeps.
#include <cmath>
#include "device_common.cuh"

namespace cmaes_gb300 {

constexpr int kJbNT = 256;
constexpr float kJbTol = 1e-6f;  // as the single-CTA FP32 Jacobi
constexpr float kJbTol2 = kJbTol * kJbTol;

__device__ __forceinline__ bool big_due(const Search& s) {
  return !s.done && s.eig_due && !s.trd && eig_big_route(s.n);
}

__host__ __device__ inline long long jb_nb(int P) { return static_cast<long long>(P) * (P - 1) / 2; }
__host__ __device__ inline long long jb_bufsz(int P) { return ((4 * jb_nb(P) + 3 * P) + 3) & ~3ll; }

// sum over d' = 3 .. d - 1 of the d'-diagonal's length P - d'
__device__ __forceinline__ long long jb_dbase(int d, int P) {
  return static_cast<long long>(d - 3) * P - (static_cast<long long>(d - 1) * d / 2 - 3);
}

// slot of off-diagonal block (K, L), K < L
__device__ __forceinline__ long long jb_slot(int K, int L, int P) {
  const int d = L - K;
  if (d == 2) return K + 1;
  if (d == 1) {
    if (K == 0) return 0;
    if (K == P - 2) return P - 1;
    return P + K - 1;
  }
  return P + (P - 3) + jb_dbase(d, P) + K;
}

// block (K, L) of slot k
__device__ __forceinline__ void jb_block(long long k, int P, int& K, int& L) {
  if (k < P) {
    if (k == 0) { K = 0; L = 1; }
    else if (k == 1) { K = 0; L = 2; }
    else if (k == P - 1) { K = P - 2; L = P - 1; }
    else { K = static_cast<int>(k) - 1; L = static_cast<int>(k) + 1; }
    return;
  }
  long long j = k - P;
  if (j < P - 3) {
    K = static_cast<int>(j) + 1;
    L = K + 1;
    return;
  }
  j -= P - 3;
  // the largest d >= 3 with jb_dbase(d) <= j: root of d^2 - (2P + 1) d + 6P - 6 + 2j = 0
  const double b = 2.0 * P + 1.0;
  const double disc = b * b - 4.0 * (6.0 * P - 6.0 + 2.0 * static_cast<double>(j));
  int d = static_cast<int>((b - sqrt(fmax(disc, 0.0))) * 0.5);
  if (d < 3) d = 3;
  while (d + 1 <= P - 1 && jb_dbase(d + 1, P) <= j) ++d;
  while (d > 3 && jb_dbase(d, P) > j) --d;
  K = static_cast<int>(j - jb_dbase(d, P));
  L = K + d;
}

// ring position (K, x) of the next step
__device__ __forceinline__ void jb_next(int K, int x, int P, int& Kn, int& xn) {
  if (x == 0) {
    Kn = K >= 1 ? K - 1 : 1;
    xn = K >= 1 ? 0 : 1;
  } else {
    Kn = (K == 0) ? 0 : (K == P - 1 ? P - 1 : K + 1);
    xn = (K == P - 1) ? 0 : 1;
  }
}

// offset of the entry between positions (K, x) and (L, y)
__device__ __forceinline__ long long jb_off(int K, int x, int L, int y, int P) {
  const long long NB = jb_nb(P);
  if (K < L) return (2 * x + y) * NB + jb_slot(K, L, P);
  if (K > L) return (2 * y + x) * NB + jb_slot(L, K, P);
  return 4 * NB + (x == y ? (x ? 2 : 0) : 1) * static_cast<long long>(P) + K;
}

__device__ __forceinline__ bool jb_rotates(float app, float aqq, float apq, float floor_abs) {
  return fabsf(apq) > floor_abs && apq * apq > kJbTol2 * fabsf(app * aqq);
}

// (c, s, t) of the rotation that annihilates a_pq (see j32_rotation)
__device__ __forceinline__ void jb_rotation(float app, float aqq, float apq, float& c, float& s, float& t) {
  const float d = aqq - app;
  const float x = fmaf(d, d, 4.f * apq * apq);
  const float h = x * rsqrtf(x);
  const float mag = __fdividef(2.f * fabsf(apq), fabsf(d) + h);
  t = (d == 0.f || ((d > 0.f) == (apq > 0.f))) ? mag : -mag;
  const float u = fmaf(t, t, 1.f);
  float y = rsqrtf(u);
  y = y * fmaf(-0.5f * u * y, y, 1.5f);
  c = y;
  s = t * y;
}

// the rotation of pair k of step t from its diagonal block (a, b, ab): new
// diagonal entries, the step record and the log entry; returns whether it
// rotates (ab is then zero)
__device__ __forceinline__ int jb_rotate_pair(Search& s, int t, int k, int P, float& a, float& b, float& ab,
                                              float2* rec) {
  float cr = 1.f, sr = 0.f;
  int act = 0;
  const bool pad = s.n & 1;  // pair 0 holds the padding element N - 1 and never rotates
  if (!(pad && k == 0) && jb_rotates(a, b, ab, s.jb_floor)) {
    float tn;
    jb_rotation(a, b, ab, cr, sr, tn);
    a -= tn * ab;
    b += tn * ab;
    ab = 0.f;
    act = 1;
  }
  rec[k] = make_float2(cr, sr);
  if (t < s.jb_tmax) reinterpret_cast<float2*>(s.jlog)[static_cast<size_t>(t) * P + k] = make_float2(cr, sr);
  if (act) atomicMax(&s.jb_last_act, t);
  return act;
}

// shift c, scale 2^-k, rounding floor and the step budget (one CTA per search)
__global__ void __launch_bounds__(1024) k_j32b_prep(Search* S, int s0) {
  __shared__ double shs[32];
  Search& s = S[s0 + blockIdx.x];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1);
  const long long L = s.ldn;
  const double* A64 = s.EH;
  double tr = 0.0, dmax = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) {
    const double d = A64[i + L * i];
    tr += d;
    dmax = fmax(dmax, fabs(d));
  }
  const double c = block_sum<1024>(tr, shs) / n;
  dmax = block_max<1024>(dmax, shs);
  int ex = 0;
  if (dmax > 0.0) frexp(dmax, &ex);
  const double scale = ldexp(1.0, -ex);  // max|a_ij - c delta_ij| <= max a_ii (B^T C B is PSD)
  double dm = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) dm = fmax(dm, fabs(A64[i + L * i] - c));
  dm = block_max<1024>(dm, shs);
  if (threadIdx.x == 0) {
    s.jb_conv = 0;
    s.jb_pend = 0;
    s.jb_done = 0;
    s.jb_shift = c;
    s.jb_scale = scale;
    s.jb_floor = 16.f * 1.1920929e-7f * static_cast<float>(dm * scale);
    s.jb_last_act = -1;
    s.jb_tmax = kJ32BigSweeps * (N - 1);
  }
}

// A32 into buffer 0 at the ring positions of step 0: element 0 at (0, a),
// N - 1 at (0, b), 1 <= e <= P - 1 at (e, a), P <= e <= N - 2 at (N - 1 - e, b)
__global__ void __launch_bounds__(kJbNT) k_j32b_load(Search* S, TileMap tm) {
  int t;
  const int si = find_search(tm, t);
  const Search& s = S[si];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2, M = N - 1;
  const long long e = static_cast<long long>(t) * kJbNT + threadIdx.x;
  if (e >= static_cast<long long>(N) * N) return;
  const int i = static_cast<int>(e % N), j = static_cast<int>(e / N);
  auto pos0 = [=](int el, int& K, int& x) {
    if (el == 0) { K = 0; x = 0; }
    else if (el == M) { K = 0; x = 1; }
    else if (el <= P - 1) { K = el; x = 0; }
    else { K = M - el; x = 1; }
  };
  int Ki, xi, Kj, xj;
  pos0(i, Ki, xi);
  pos0(j, Kj, xj);
  if (!(Ki < Kj || (Ki == Kj && xi <= xj))) return;  // each unordered entry once
  float v = 0.f;
  if (i < n && j < n)
    v = static_cast<float>((s.EH[i + s.ldn * j] - (i == j ? s.jb_shift : 0.0)) * s.jb_scale);
  s.jb_buf[jb_off(Ki, xi, Kj, xj, P)] = v;
}

// the rotations of step 0 from the diagonal blocks of buffer 0
__global__ void __launch_bounds__(1024) k_j32b_first(Search* S, int s0) {
  Search& s = S[s0 + blockIdx.x];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2;
  float* D = s.jb_buf + 4 * jb_nb(P);
  float2* rec = reinterpret_cast<float2*>(s.jb_rec);
  for (int k = threadIdx.x; k < P; k += 1024) {
    float a = D[k], ab = D[P + k], b = D[2 * P + k];
    jb_rotate_pair(s, 0, k, P, a, b, ab, rec);
    D[k] = a;
    D[P + k] = ab;
    D[2 * P + k] = b;
  }
}

// step t: the blocks with the rotations of step t, written to step t + 1's
// positions; the role threads form the rotations of step t + 1
__global__ void __launch_bounds__(kJbNT) k_j32b_step(Search* S, TileMap tm, int t) {
  int tile;
  const int si = find_search(tm, tile);
  Search& s = S[si];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2, M = N - 1;
  if (s.jb_conv || t >= s.jb_tmax || t - s.jb_last_act >= M) return;  // converged or budget spent
  const long long NB = jb_nb(P), k = static_cast<long long>(tile) * kJbNT + threadIdx.x;
  if (k >= NB) return;
  const long long bsz = jb_bufsz(P);
  const float* bc = s.jb_buf + (t & 1) * bsz;
  float* bn = s.jb_buf + ((t + 1) & 1) * bsz;
  const float2* rc = reinterpret_cast<const float2*>(s.jb_rec) + (t & 1) * P;
  float2* rn = reinterpret_cast<float2*>(s.jb_rec) + ((t + 1) & 1) * P;
  int K, L;
  jb_block(k, P, K, L);
  float x[4] = {bc[k], bc[NB + k], bc[2 * NB + k], bc[3 * NB + k]};
  const float2 gK = rc[K], gL = rc[L];
  if (gK.y != 0.f || gL.y != 0.f) {
    const float cP = gK.x, sP = gK.y, cQ = gL.x, sQ = gL.y;
    const float y00 = x[0] * cQ - x[1] * sQ, y01 = x[0] * sQ + x[1] * cQ;
    const float y10 = x[2] * cQ - x[3] * sQ, y11 = x[2] * sQ + x[3] * cQ;
    x[0] = cP * y00 - sP * y10;
    x[1] = cP * y01 - sP * y11;
    x[2] = sP * y00 + cP * y10;
    x[3] = sP * y01 + cP * y11;
  }
  if (k < P) {
    // next-step pair kk = k: its pivot is entry ent of this block, its
    // diagonal entries sit at (kk + 1, a) (or (P - 1, b)) and (kk - 1, b)
    // (or (0, a), (0, b)) of this step, finished in the step before
    const int kk = static_cast<int>(k);
    const int ent = kk == 1 ? 0 : (kk == P - 1 ? 3 : 2);
    const float* D = bc + 4 * NB;
    float a = kk <= P - 2 ? D[kk + 1] : D[2 * P + P - 1];
    float b = kk >= 2 ? D[2 * P + kk - 1] : (kk == 1 ? D[0] : D[2 * P]);
    float ab = ent == 0 ? x[0] : (ent == 2 ? x[2] : x[3]);
    jb_rotate_pair(s, t + 1, kk, P, a, b, ab, rn);
    if (ent == 0) x[0] = ab;
    else if (ent == 2) x[2] = ab;
    else x[3] = ab;
    float* Dn = bn + 4 * NB;
    Dn[kk] = a;
    Dn[2 * P + kk] = b;
    // the current diagonal block kk's a_ab moves on with the ring
    int Ka, xa, Kb, xb;
    jb_next(kk, 0, P, Ka, xa);
    jb_next(kk, 1, P, Kb, xb);
    bn[jb_off(Ka, xa, Kb, xb, P)] = D[P + kk];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int Kn, xn, Ln, yn;
    jb_next(K, e >> 1, P, Kn, xn);
    jb_next(L, e & 1, P, Ln, yn);
    bn[jb_off(Kn, xn, Ln, yn, P)] = x[e];
  }
}

// Whole-matrix check before step t (buffer t & 1 holds the matrix of step t,
// with step t's diagonal blocks already rotated): when step t rotates nothing
// the buffer is the current matrix, and if no off-diagonal entry passes the
// test either, the search has converged.
__global__ void __launch_bounds__(kJbNT) k_j32b_check(Search* S, TileMap tm, int t) {
  __shared__ int sh_pend;
  int tile;
  const int si = find_search(tm, tile);
  Search& s = S[si];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2, M = N - 1;
  // uniform over the search's CTAs: the fields are only written by the
  // step kernels before this launch and by the deciding CTA at its very end
  if (s.jb_conv || t >= s.jb_tmax || t - s.jb_last_act >= M || s.jb_last_act >= t) return;
  const long long NB = jb_nb(P), k = static_cast<long long>(tile) * kJbNT + threadIdx.x;
  const float* bc = s.jb_buf + (t & 1) * jb_bufsz(P);
  const float* D = bc + 4 * NB;
  if (threadIdx.x == 0) sh_pend = 0;
  __syncthreads();
  int pend = 0;
  if (k < NB) {
    int K, L;
    jb_block(k, P, K, L);
    const float aK = D[K], bK = D[2 * P + K], aL = D[L], bL = D[2 * P + L];
    const float fl = s.jb_floor;
    pend = jb_rotates(aK, aL, bc[k], fl) | jb_rotates(aK, bL, bc[NB + k], fl) |
           jb_rotates(bK, aL, bc[2 * NB + k], fl) | jb_rotates(bK, bL, bc[3 * NB + k], fl);
    if (k < P) pend |= jb_rotates(D[k], D[2 * P + k], D[P + k], fl);
  }
  if (pend) sh_pend = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sh_pend) atomicOr(&s.jb_pend, 1);
    __threadfence();
    const int ntile = static_cast<int>((NB + kJbNT - 1) / kJbNT);
    if (atomicAdd(&s.jb_done, 1) == ntile - 1) {  // the last CTA of this search decides
      __threadfence();
      if (atomicOr(&s.jb_pend, 0) == 0) s.jb_conv = 1;
      s.jb_pend = 0;
      s.jb_done = 0;
    }
  }
}

// V32 from the log (T = last rotating step + 1 steps; step t has r = t mod
// (N - 1)): one warp per row, kJrRows rows per CTA in shared memory, the log
// staged in shared memory in chunks of whole steps shared by the CTA's rows.
// Rows leave as FP64 into EG.
constexpr int kJrRows = 8;
constexpr int kJrNT = kJrRows * 32;
constexpr int kJrChunk = 4096;  // (c, s) entries per chunk

__global__ void __launch_bounds__(kJrNT) k_jlog_big(Search* S, TileMap tm) {
  extern __shared__ __align__(16) float jsm[];
  int tile;
  const int si = find_search(tm, tile);
  Search& s = S[si];
  if (!big_due(s)) return;
  const int n = s.n, N = n + (n & 1), P = N / 2, M = N - 1;
  const int i0 = tile * kJrRows;
  if (i0 >= n) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, i = i0 + warp;
  float2* lcs = reinterpret_cast<float2*>(jsm);  // 2 x kJrChunk
  float* vrow = jsm + 4 * kJrChunk;              // kJrRows x (N + 1)
  float* v = vrow + warp * (N + 1);
  for (int j = lane; j < N; j += 32) v[j] = (j == i) ? 1.f : 0.f;
  int T = s.jb_last_act + 1;
  if (T > s.jb_tmax) T = s.jb_tmax;
  const int K = kJrChunk / P;  // steps per chunk (P <= 2048 for n <= 4096: at least 2)
  const int nch = ceil_div(T, K);
  const float2* jlog = reinterpret_cast<const float2*>(s.jlog);
  for (int c = 0; c < nch; ++c) {
    const int t0 = c * K, cnt = min(K, T - t0);
    float2* buf = lcs + (c & 1) * kJrChunk;
    // the other buffer was last read in chunk c - 1, before the barrier that ended it
    for (int e = tid; e < cnt * P; e += kJrNT) buf[e] = __ldg(jlog + static_cast<size_t>(t0) * P + e);
    __syncthreads();
    for (int kk = 0; kk < cnt; ++kk) {
      const int r = (t0 + kk) % M;
      const float2* g = buf + kk * P;
      for (int pi = lane; pi < P; pi += 32) {
        const float2 cs = g[pi];
        if (cs.y == 0.f) continue;  // identity
        int p = r + pi, q = r - pi;
        if (p >= M) p -= M;
        if (q < 0) q += M;
        if (pi == 0) q = M;
        const float x = v[p], y = v[q];
        v[p] = cs.x * x - cs.y * y;
        v[q] = cs.y * x + cs.x * y;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  const long long L = s.ldn;
  const int rows = min(kJrRows, n - i0);
  for (int e = tid; e < kJrRows * n; e += kJrNT) {
    const int ii = e % kJrRows, j = e / kJrRows;
    if (ii < rows) s.EG[(i0 + ii) + L * j] = static_cast<double>(vrow[ii * (N + 1) + j]);
  }
  if (tile == 0 && tid == 0) s.eig_sweeps32 += ceil_div(T, M);
}

int tiles_jb_blocks(int n) {
  if (!eig_big_route(n)) return 0;
  const int P = (n + (n & 1)) / 2;
  return static_cast<int>((jb_nb(P) + kJbNT - 1) / kJbNT);
}
int tiles_jb_load(int n) {
  if (!eig_big_route(n)) return 0;
  const long long N = n + (n & 1);
  return static_cast<int>((N * N + kJbNT - 1) / kJbNT);
}
int tiles_jb_rows(int n) { return eig_big_route(n) ? ceil_div(n, kJrRows) : 0; }
size_t jb_buf_floats(int n) {
  const int P = (n + (n & 1)) / 2;
  return static_cast<size_t>(2 * jb_bufsz(P));
}

void launch_j32b_start(Search* S, TileMap tload, int s0, int s1, cudaStream_t st) {
  if (s1 <= s0) return;
  k_j32b_prep<<<s1 - s0, 1024, 0, st>>>(S, s0);
  if (tload.total > 0) k_j32b_load<<<tload.total, kJbNT, 0, st>>>(S, tload);
  k_j32b_first<<<s1 - s0, 1024, 0, st>>>(S, s0);
}

void launch_j32b_step(Search* S, TileMap tblk, int t, cudaStream_t st) {
  if (tblk.total > 0) k_j32b_step<<<tblk.total, kJbNT, 0, st>>>(S, tblk, t);
}

void launch_j32b_check(Search* S, TileMap tblk, int t, cudaStream_t st) {
  if (tblk.total > 0) k_j32b_check<<<tblk.total, kJbNT, 0, st>>>(S, tblk, t);
}

void launch_jlog_big(Search* S, TileMap trows, int max_n, cudaStream_t st) {
  if (trows.total <= 0) return;
  const int N = max_n + (max_n & 1);
  const int bytes = 2 * kJrChunk * 8 + kJrRows * (N + 1) * 4;
  cudaFuncSetAttribute(k_jlog_big, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  k_jlog_big<<<trows.total, kJrNT, bytes, st>>>(S, trows);
}

}  // namespace cmaes_gb300
