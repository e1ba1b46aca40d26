// kernels_eig_trd_bt.cu -- back-transformation B = Q V of the tridiagonal
// route with the reflectors blocked (the compact WY form of Schreiber and
// Van Loan, 1989) and every product on the tensor cores in FP64-accurate
// digit-plane form (ozaki.cuh).
//
// Q = H_0 H_1 ... H_{n-2}, H_k = I - tau_k v_k v_k^T, v_k (rows k+1.., unit
// first entry) in column k of EX. Panel p gathers the 128 reflectors from
// k0 = 128 p: H_k0 ... H_k0+nb-1 = I - Y_p T_p Y_p^T with Y_p the seg_p x nb
// reflector block (rows k0 + 1 ..) and T_p upper triangular,
//   T(c, c) = tau_c,  T(0:c, c) = -tau_c T(0:c, 0:c) (Y_p^T Y_p)(0:c, c).
// B = Q_0 (Q_1 (... (Q_{P-1} V))): the panels are applied last to first, each
// as three products on the rows below k0:
//   W = Y_p^T V,   W' = T_p W,   V <- V - Y_p W'.
// Setup (independent of V): Y_p^T and Y_p as packed operands, the Gram
// Y_p^T Y_p, T_p and its packed form, for every panel at once. Then one step
// per panel, batched over the searches (each at its own panel). Last, the
// canonical column sign and the ascending eigenvalue order.
#include <cmath>
#include "device_common.cuh"
#include "ozaki.cuh"
#include "trd_common.cuh"

namespace cmaes_gb300 {

constexpr int kBtFinCols = 8;  // columns per CTA of the final pass (one warp each)

int tiles_bt_pack(int n) {
  if (!trd_bt_blocked(n)) return 0;
  int t = 2 * trd_panels(n);
  for (int p = 0; p < trd_panels(n); ++p) t += oz_rows_padded(trd_seg(n, p)) / 64;
  return t;
}
int tiles_bt_gram(int n) { return trd_bt_blocked(n) ? 2 * trd_panels(n) : 0; }
int tiles_bt_tfac(int n) { return trd_bt_blocked(n) ? trd_panels(n) : 0; }
int tiles_bt_rows(int n) { return trd_bt_blocked(n) ? oz_rows_padded(n) / 64 : 0; }
int tiles_bt_cols(int n) { return trd_bt_blocked(n) ? ceil_div(n, kOzBN) : 0; }
int tiles_bt_update(int n) { return trd_bt_blocked(n) ? ceil_div(n - 1, kOzBM) * ceil_div(n, kOzBN) : 0; }
int tiles_bt_final(int n) { return trd_bt_blocked(n) ? ceil_div(n, kBtFinCols) : 0; }
static size_t bt_tfac_smem() { return static_cast<size_t>(kBtNb) * kBtNb * 8; }

// ---------------------------------------------------------------- setup ----
// Tiles 0 .. 2P-1: the two 64-row blocks of Y_p^T (row c = reflector k0 + c,
// K = seg_p rows); then the 64-row blocks of every Y_p (row r = matrix row
// k0 + 1 + r, K = 128 reflectors).
__global__ void __launch_bounds__(kOzNT) k_bt_pack_y(Search* S, TileMap tm) {
  __shared__ int sh_e[64];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, P = trd_panels(n);
  const TrdOz lay = trd_oz_layout(n);
  const long long L = s.ldn;
  const double* X = s.EX;
  if (tile < 2 * P) {
    const int p = tile >> 1, k0 = kBtNb * p, seg = trd_seg(n, p), nb = trd_panel_nb(n, p);
    oz_pack_block_get(
        [=] __device__(int c, int k) { return (c < nb && k >= c) ? X[(k0 + 1 + k) + L * (k0 + c)] : 0.0; }, true,
        kBtNb, seg, tile & 1, oz_nks(seg), s.ozp + lay.yt + trd_oz_yt_off(n, p), s.oze + lay.eyt + kBtNb * p, sh_e);
    return;
  }
  int t = tile - 2 * P, p = 0;
  while (p < P - 1 && t >= oz_rows_padded(trd_seg(n, p)) / 64) {
    t -= oz_rows_padded(trd_seg(n, p)) / 64;
    ++p;
  }
  const int k0 = kBtNb * p, seg = trd_seg(n, p), nb = trd_panel_nb(n, p);
  oz_pack_block_get(
      [=] __device__(int r, int c) { return (c < nb && r >= c) ? X[(k0 + 1 + r) + L * (k0 + c)] : 0.0; }, false,
      seg, kBtNb, t, oz_nks(kBtNb), s.ozp + lay.y + trd_oz_y_off(n, p), s.oze + lay.ey + trd_oz_ey_off(n, p), sh_e);
}

// G_p = Y_p^T Y_p, columns 64 h .. 64 h + 63 (tile 2 p + h).
__global__ void __launch_bounds__(kOzNT, 1) k_bt_gram(Search* S, TileMap tm) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, p = tile >> 1, h = tile & 1, seg = trd_seg(n, p);
  const TrdOz lay = trd_oz_layout(n);
  const unsigned char* yt = s.ozp + lay.yt + trd_oz_yt_off(n, p);
  const int* e = s.oze + lay.eyt + kBtNb * p;
  double* G = reinterpret_cast<double*>(s.ozp + lay.g) + static_cast<size_t>(p) * kBtNb * kBtNb;
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long Wq[32];
  float Lq[32];
  const long long pitch = oz_pitch(oz_nks(seg));
  const bool ok = oz_tile(cx, yt, pitch, 0, yt, pitch, h, oz_nks(seg), Wq, Lq);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 3) + lane, jb = kOzBN * h + 32 * (warp >> 2);
  if (ok) {
    const int ei = e[i];
#pragma unroll
    for (int q = 0; q < 32; ++q) G[i + kBtNb * (jb + q)] = oz_value(Wq[q], Lq[q], ei, e[jb + q]);
  } else if (threadIdx.x == 0) {
    atomicOr(s.err, kDevErrTimeout);
  }
  oz_end(cx);
}

// T_p (column by column in shared memory; row r of every column is formed by
// thread r from its own earlier entries) and its packed form.
__global__ void __launch_bounds__(kOzNT) k_bt_tfac(Search* S, TileMap tm) {
  extern __shared__ double Tsm[];  // 128 x 128, column-major
  __shared__ int sh_e[64];
  int p;
  const int si = find_search(tm, p);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, k0 = kBtNb * p, nb = trd_panel_nb(n, p);
  const TrdOz lay = trd_oz_layout(n);
  const double* G = reinterpret_cast<const double*>(s.ozp + lay.g) + static_cast<size_t>(p) * kBtNb * kBtNb;
  double* Tg = reinterpret_cast<double*>(s.ozp + lay.tf) + static_cast<size_t>(p) * kBtNb * kBtNb;
  const double* tau = tv(s, TV_TAU);
  for (int e = threadIdx.x; e < kBtNb * kBtNb; e += kOzNT) Tsm[e] = 0.0;
  __syncthreads();
  const int r = threadIdx.x;
  for (int c = 0; c < kBtNb; ++c) {
    const double tc = c < nb ? tau[k0 + c] : 0.0;
    if (r < c) {
      double acc = 0.0;
      for (int l = r; l < c; ++l) acc = fma(Tsm[r + kBtNb * l], G[l + kBtNb * c], acc);
      Tsm[r + kBtNb * c] = -tc * acc;
    } else if (r == c) {
      Tsm[c + kBtNb * c] = tc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBtNb * kBtNb; e += kOzNT) Tg[e] = Tsm[e];
  unsigned char* out = s.ozp + lay.t + static_cast<size_t>(p) * trd_align256(oz_bytes(kBtNb, kBtNb));
  int* eo = s.oze + lay.et + kBtNb * p;
  for (int rb = 0; rb < 2; ++rb) {
    oz_pack_block_get([=] __device__(int i, int k) { return Tsm[i + kBtNb * k]; }, false, kBtNb, kBtNb, rb,
                      oz_nks(kBtNb), out, eo, sh_e);
    __syncthreads();
  }
}

// ------------------------------------------------------------ one panel ----
// The panel that step `step` applies for search s (-1: none left).
__device__ __forceinline__ int bt_panel(const Search& s, int step) { return trd_panels(s.n) - 1 - step; }

// The columns of V (rows k0 + 1 .. n - 1 of EA) as the rows of a packed
// operand with K = seg_p.
__global__ void __launch_bounds__(kOzNT) k_bt_pack_v(Search* S, TileMap tm, int step) {
  __shared__ int sh_e[64];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int p = bt_panel(s, step);
  if (p < 0) return;
  const int n = s.n, k0 = kBtNb * p, seg = trd_seg(n, p);
  const TrdOz lay = trd_oz_layout(n);
  const long long L = s.ldn;
  const double* V = s.EA;
  oz_pack_block_get([=] __device__(int j, int k) { return V[(k0 + 1 + k) + L * j]; }, true, n, seg, tile,
                    oz_nks(seg), s.ozp + lay.v, s.oze + lay.ev, sh_e);
}

// The columns of W (128 x n, FP64) as the rows of a packed operand, K = 128.
__global__ void __launch_bounds__(kOzNT) k_bt_pack_w(Search* S, TileMap tm, int step) {
  __shared__ int sh_e[64];
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s) || bt_panel(s, step) < 0) return;
  const int n = s.n;
  const TrdOz lay = trd_oz_layout(n);
  const double* Wf = reinterpret_cast<const double*>(s.ozp + lay.wf);
  oz_pack_block_get([=] __device__(int j, int c) { return Wf[c + kBtNb * j]; }, true, n, kBtNb, tile,
                    oz_nks(kBtNb), s.ozp + lay.w, s.oze + lay.ew, sh_e);
}

// which = 0: W = Y_p^T V (A = packed Y_p^T, B = packed V, K = seg_p);
// which = 1: W' = T_p W  (A = packed T_p,  B = packed W, K = 128).
// One 128 x 64 tile of the 128 x n result per CTA, into wf.
__global__ void __launch_bounds__(kOzNT, 1) k_bt_small(Search* S, TileMap tm, int step, int which) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int p = bt_panel(s, step);
  if (p < 0) return;
  const int n = s.n, seg = trd_seg(n, p);
  const TrdOz lay = trd_oz_layout(n);
  const unsigned char* A;
  const unsigned char* B;
  const int *ea, *eb;
  int nks;
  if (which == 0) {
    A = s.ozp + lay.yt + trd_oz_yt_off(n, p);
    ea = s.oze + lay.eyt + kBtNb * p;
    B = s.ozp + lay.v;
    eb = s.oze + lay.ev;
    nks = oz_nks(seg);
  } else {
    A = s.ozp + lay.t + static_cast<size_t>(p) * trd_align256(oz_bytes(kBtNb, kBtNb));
    ea = s.oze + lay.et + kBtNb * p;
    B = s.ozp + lay.w;
    eb = s.oze + lay.ew;
    nks = oz_nks(kBtNb);
  }
  double* Wf = reinterpret_cast<double*>(s.ozp + lay.wf);
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long Wq[32];
  float Lq[32];
  const long long pitch = oz_pitch(nks);
  const bool ok = oz_tile(cx, A, pitch, 0, B, pitch, tile, nks, Wq, Lq);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 3) + lane, jb = kOzBN * tile + 32 * (warp >> 2);
  if (ok) {
    const int ei = ea[i];
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (jb + q < n) Wf[i + kBtNb * (jb + q)] = oz_value(Wq[q], Lq[q], ei, eb[jb + q]);
  } else if (threadIdx.x == 0) {
    atomicOr(s.err, kDevErrTimeout);
  }
  oz_end(cx);
}

// V(k0 + 1 + i, j) -= (Y_p W')(i, j): A = packed Y_p (row block pair 2 mt),
// B = packed W' (row block nt), K = 128.
__global__ void __launch_bounds__(kOzNT, 1) k_bt_update(Search* S, TileMap tm, int step) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  int tile;
  const int si = find_search(tm, tile);
  const Search& s = S[si];
  if (!trd_due(s)) return;
  const int p = bt_panel(s, step);
  if (p < 0) return;
  const int n = s.n, k0 = kBtNb * p, seg = trd_seg(n, p);
  const int TN = ceil_div(n, kOzBN), mt = tile / TN, nt = tile % TN;
  if (mt * kOzBM >= seg) return;
  const TrdOz lay = trd_oz_layout(n);
  const unsigned char* A = s.ozp + lay.y + trd_oz_y_off(n, p);
  const int* ea = s.oze + lay.ey + trd_oz_ey_off(n, p);
  const int* eb = s.oze + lay.ew;
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long Wq[32];
  float Lq[32];
  const long long pitch = oz_pitch(oz_nks(kBtNb));
  const bool ok = oz_tile(cx, A, pitch, 2 * mt, s.ozp + lay.w, pitch, nt, oz_nks(kBtNb), Wq, Lq);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = kOzBM * mt + 32 * (warp & 3) + lane, jb = kOzBN * nt + 32 * (warp >> 2);
  if (ok) {
    if (i < seg) {
      const int ei = ea[i];
      const long long L = s.ldn;
      double* V = s.EA + (k0 + 1 + i);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = jb + q;
        if (j < n) V[L * j] -= oz_value(Wq[q], Lq[q], ei, eb[j]);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(s.err, kDevErrTimeout);
  }
  oz_end(cx);
}

// Column t of Q V (in EA) to column rank[t] of B with the entry of largest
// magnitude (the first on ties) positive; one warp per column.
__global__ void __launch_bounds__(kTrdNT) k_bt_final(Search* S, TileMap tm) {
  int tile;
  const int si = find_search(tm, tile);
  Search& s = S[si];
  if (!trd_due(s)) return;
  const int n = s.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = tile * kBtFinCols + warp;
  if (warp >= kBtFinCols || t >= n) return;  // whole warps leave
  const long long L = s.ldn;
  const double* x = s.EA + L * t;
  double best = -1.0, val = 0.0;
  int bi = 0x7fffffff;
  for (int i = lane; i < n; i += 32) {
    const double a = fabs(x[i]);
    if (a > best) {
      best = a;
      val = x[i];
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
  for (int i = lane; i < n; i += 32) Bc[i] = sg * x[i];
}

// ------------------------------------------------------------------ host ----
void bt_set_attributes() {
  cudaFuncSetAttribute(k_bt_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  cudaFuncSetAttribute(k_bt_small, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  cudaFuncSetAttribute(k_bt_update, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  cudaFuncSetAttribute(k_bt_tfac, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bt_tfac_smem()));
}

int launch_bt(Search* S, const TrdMaps& m, int max_n, cudaStream_t st) {
  int nl = 0;
  auto go = [&](const TileMap& t) { return t.total > 0 ? (++nl, true) : false; };
  if (go(m.btpack)) k_bt_pack_y<<<m.btpack.total, kOzNT, 0, st>>>(S, m.btpack);
  if (go(m.btgram)) k_bt_gram<<<m.btgram.total, kOzNT, kOzSmem, st>>>(S, m.btgram);
  if (go(m.bttfac)) k_bt_tfac<<<m.bttfac.total, kOzNT, bt_tfac_smem(), st>>>(S, m.bttfac);
  const int steps = trd_bt_blocked(max_n) ? trd_panels(max_n) : 0;
  for (int r = 0; r < steps; ++r) {
    if (go(m.btrows)) k_bt_pack_v<<<m.btrows.total, kOzNT, 0, st>>>(S, m.btrows, r);
    if (go(m.btcols)) k_bt_small<<<m.btcols.total, kOzNT, kOzSmem, st>>>(S, m.btcols, r, 0);
    if (go(m.btrows)) k_bt_pack_w<<<m.btrows.total, kOzNT, 0, st>>>(S, m.btrows, r);
    if (go(m.btcols)) k_bt_small<<<m.btcols.total, kOzNT, kOzSmem, st>>>(S, m.btcols, r, 1);
    if (go(m.btrows)) k_bt_pack_w<<<m.btrows.total, kOzNT, 0, st>>>(S, m.btrows, r);
    if (go(m.btupd)) k_bt_update<<<m.btupd.total, kOzNT, kOzSmem, st>>>(S, m.btupd, r);
  }
  if (go(m.btfin)) k_bt_final<<<m.btfin.total, kTrdNT, 0, st>>>(S, m.btfin);
  return nl;
}

}  // namespace cmaes_gb300
