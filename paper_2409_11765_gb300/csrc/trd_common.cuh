// trd_common.cuh -- state shared by the kernels of the tridiagonal route of
// the eigendecomposition (kernels_eig_trd.cu, kernels_eig_trd_bt.cu): the
// per-search scratch vectors and the layout of the packed operands of its
// FP64-accurate tensor-core products.
#pragma once
#include "device_common.cuh"
#include "ozaki.cuh"

namespace cmaes_gb300 {

// --------------------------------------------------------------------------
// Scratch of one search (Search::trd_v: TV_COUNT vectors of ldn doubles,
// Search::trd_i: TI_COUNT vectors of ldn ints) and its matrices: W (the matrix
// being reduced) = EA, reflectors = EX (column k holds v_k in rows k+1..),
// eigenvectors of T = ET (column t), inverse-iteration factors = EA, EG, EH
// (after the reduction), I - V^T V in FP32 = EG, the Newton-Schulz iterates
// alternate between ET and EA and end in EA.
// --------------------------------------------------------------------------
enum { TV_D = 0, TV_E, TV_ES, TV_E2, TV_TAU, TV_LAMB, TV_LAMS, TV_P0, TV_P1, TV_SD, TV_SCAL };
enum { TI_B0 = 0, TI_B1, TI_RANK, TI_CL0, TI_TFLAG };
// scalars at TV_SCAL: ||T|| bound, pivmin, split threshold, cluster threshold,
// and the orthogonality defect max |(I - V^T V) / 2| before each Newton-Schulz
// step (as ordered bit patterns for atomicMax)
constexpr double kTrdSplit = 4.0;
constexpr double kTrdClus = 1e-13;
constexpr int kTrdClusMax = 64;      // Gram-Schmidt chunk of a longer cluster
constexpr int kTrdNsSteps = 3;
constexpr double kTrdNsSkip = 5e-9;  // one step leaves 1.5 (2 * 5e-9)^2 < eps64
// V^T V is formed only for 64 x 64 tiles holding a pair of vectors of one
// block whose eigenvalues lie within kTrdNsBand ||T||: for a pair further apart
// inverse iteration already leaves |v_i^T v_j| <~ eps64 / kTrdNsBand ~ 1e-14.
constexpr double kTrdNsBand = 1e-2;
constexpr double kTrdEps = 0x1p-53;
constexpr long long kTrdWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr int kTrdNT = 256;

__device__ __forceinline__ bool trd_due(const Search& s) { return s.trd && !s.done && s.eig_due; }

__device__ __forceinline__ double* tv(const Search& s, int which) {
  return s.trd_v + static_cast<long long>(which) * s.ldn;
}
__device__ __forceinline__ int* ti(const Search& s, int which) {
  return s.trd_i + static_cast<long long>(which) * s.ldn;
}

// --------------------------------------------------------------------------
// Search::ozp, byte offsets (each 256-aligned), for an n x n problem with
// P = ceil((n - 1) / 128) panels of reflectors (panel p: reflectors 128 p ..,
// acting on the seg_p = n - 128 p - 1 rows below 128 p):
//   v   the columns of V as a packed operand (K = n or seg_p)
//   yt  per panel, its reflectors as the rows of a packed operand (K = seg_p)
//   y   per panel, the rows of its reflector block (K = 128)
//   t   per panel, the rows of its triangular factor T_p (K = 128)
//   w   the columns of W = Y_p^T V (or T_p W) as a packed operand (K = 128)
//   g, tf  per panel, Y_p^T Y_p and T_p in FP64 (128 x 128, column-major)
//   wf  W in FP64 (128 x n, column-major)
//   s2a, s2b  the reduction's trailing update: [V W] and [W V] (K = 2 kPnb)
// Search::oze, int offsets: v [0, np), w [np, 2 np), yt 2 np + 128 p,
// y 2 np + 128 P + (padded rows of the earlier panels), t after y (128 per
// panel), with np the padded n.
// --------------------------------------------------------------------------
constexpr int kBtNb = 128;  // reflectors per panel of the back-transformation
constexpr int kPnb = kTrdPanel;  // columns per panel of the reduction
constexpr int kPartStride = 2 * kPnb + 8;  // per-CTA partial sums of a reduction step
// Back-transformation: blocked on the tensor cores from this size on, one
// register-resident column per warp in FP64 below it. The launches of the
// blocked form are shared by every search of a batch, so in a large batch it
// wins from n ~ 256 on (the 256-search batch: 146 -> 127 ms per generation
// when its n = 500 searches moved to it); a lone n = 300 search is ~0.2 ms
// slower in it than in the register form.
constexpr int kBtBlockedMinN = 257;
__host__ __device__ inline bool trd_bt_blocked(int n) { return n >= kBtBlockedMinN; }

__host__ __device__ inline size_t trd_align256(size_t b) { return (b + 255) / 256 * 256; }
__host__ __device__ inline int trd_panels(int n) { return n > 1 ? (n - 1 + kBtNb - 1) / kBtNb : 0; }
__host__ __device__ inline int trd_seg(int n, int p) { return n - kBtNb * p - 1; }
__host__ __device__ inline int trd_panel_nb(int n, int p) {
  const int r = (n - 1) - kBtNb * p;
  return r < kBtNb ? r : kBtNb;
}

struct TrdOz {
  size_t v, yt, y, t, w, g, tf, wf, s2a, s2b, total;  // bytes
  int ev, ew, eyt, ey, et, etotal;         // ints
};

__host__ __device__ inline TrdOz trd_oz_layout(int n) {
  TrdOz L;
  const int P = trd_panels(n), np = oz_rows_padded(n);
  size_t o = 0;
  L.v = o;
  o += trd_align256(oz_bytes(n, n));
  L.yt = o;
  for (int p = 0; p < P; ++p) o += trd_align256(oz_bytes(kBtNb, trd_seg(n, p)));
  L.y = o;
  for (int p = 0; p < P; ++p) o += trd_align256(oz_bytes(trd_seg(n, p), kBtNb));
  L.t = o;
  o += static_cast<size_t>(P) * trd_align256(oz_bytes(kBtNb, kBtNb));
  L.w = o;
  o += trd_align256(oz_bytes(n, kBtNb));
  L.g = o;
  o += static_cast<size_t>(P) * kBtNb * kBtNb * 8;
  L.tf = o;
  o += static_cast<size_t>(P) * kBtNb * kBtNb * 8;
  L.wf = o;
  o += trd_align256(static_cast<size_t>(kBtNb) * n * 8);
  L.s2a = o;
  o += trd_align256(oz_bytes(n, 2 * kPnb));
  L.s2b = o;
  o += trd_align256(oz_bytes(n, 2 * kPnb));
  L.total = o;
  int e = 0;
  L.ev = e;
  e += np;
  L.ew = e;
  e += np;
  L.eyt = e;
  e += kBtNb * P;
  L.ey = e;
  for (int p = 0; p < P; ++p) e += oz_rows_padded(trd_seg(n, p));
  L.et = e;
  e += kBtNb * P;
  L.etotal = e;
  return L;
}
// per-panel offsets inside yt and y (bytes) and inside the y exponents (ints)
__host__ __device__ inline size_t trd_oz_yt_off(int n, int p) {
  size_t o = 0;
  for (int q = 0; q < p; ++q) o += trd_align256(oz_bytes(kBtNb, trd_seg(n, q)));
  return o;
}
__host__ __device__ inline size_t trd_oz_y_off(int n, int p) {
  size_t o = 0;
  for (int q = 0; q < p; ++q) o += trd_align256(oz_bytes(trd_seg(n, q), kBtNb));
  return o;
}
__host__ __device__ inline int trd_oz_ey_off(int n, int p) {
  int o = 0;
  for (int q = 0; q < p; ++q) o += oz_rows_padded(trd_seg(n, q));
  return o;
}

}  // namespace cmaes_gb300
