// engine.h -- device data layout and kernel launchers of the batched engine.
//
// Every search owns a slice of one device arena. Vectors are padded to
// ldn = round_up(n, 16) doubles; matrices are ldn x n column-major; population
// panels are ldn x lam_cap column-major (one candidate per column), so a
// column starts on a 128-byte boundary.
#pragma once
#include <cstddef>
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace cmaes_gb300 {

constexpr int kPhaseSample = 0;
constexpr int kPhaseObjective = 1;
constexpr int kPhaseUpdate = 2;
constexpr int kPhaseCov = 3;
constexpr int kPhaseEig = 4;
constexpr int kPhaseStop = 5;
constexpr int kNumPhases = 6;

// Options shared by all searches of one handle (passed by value to kernels).
struct DevOptions {
  int max_restarts;
  int ipop_double;
  int eig_every;
  int max_iter;
  int stop_mask;
  int precision;
  int restart_hold;  // 1: a stopped descent pauses (done = 2) until the host restarts it
  double f_target;
  double box_lo, box_hi;
  double tol_hist_fun, tol_x_factor, cond_max;
  uint32_t key0, key1;  // Philox key (seed)
};

// TolHistFun on a mixed handle: the window's range of best f is compared with
// at least this multiple of the largest |f_mixed - f_FP64| of its best points
// (Search::hist holds the best values, then those errors, hist_cap apart).
constexpr double kMixedResolution = 10.0;

// Per-search descriptor, resident in device memory. Constant part first,
// then the scalars that the kernels update every generation.
// Bits of the device status word (Search::err): a bounded device wait gave up
// (reported as CMAES_ETIMEOUT, sticky), a search's state became non-finite
// (reported once as CMAES_ENUMERIC; the stop test restarts or ends the search).
constexpr int kDevErrTimeout = 1;
constexpr int kDevErrNonFinite = 2;

struct Search {
  // --- constant after create ---
  int n, ldn, lam0, lam_cap, mu_cap, hist_cap, index, obj;
  double sigma0;
  double *m, *ps, *pc, *D, *xstar, *lamdiag, *best_x, *yw, *zw, *w, *hist;
  double *part;                      // partial sums of the two-stage reductions
  double *covpart;                   // rank-mu partial tiles: tiles_sym x cov_nch x 64 x 64
  int cov_kc, cov_nch;               // rank chunk length and chunk count of the split
  double *C, *B, *BD, *Q, *EA, *ET;  // ldn x n (EA, ET: eigensolver scratch)
  double *Z, *Y, *X, *U, *f;         // ldn x lam_cap (f: lam_cap)
  int *order, *rank;                 // lam_cap
  // --- mutable ---
  double sigma, best_f, mueff, cs, ds, cc, c1, cmu, chin, psnorm, hsig;
  int lam, mu, gen, restart, g_eig, hist_len, max_iter, hist_count;
  int done, flags, eig_due, eig_sweeps, pad_;
  // eigensolver work counters (decompositions, FP64 sweeps, rotations applied,
  // FP32 sweeps of the mixed-precision route)
  long long eig_count, eig_sweeps_total, eig_rotations, eig_sweeps32;
  // mixed precision (precision != FP64): tensor-core operands, K padded to kp
  int mixed, kp, covm_kc, covm_nch;
  void *BDT;          // n x kp, row i = (B diag(D))(i, :), input format (TF32 / BF16)
  void *QTh, *QTl;    // n x kp, row i = Q(i, :), hi and lo parts
  float *lam32;       // n: Lambda in FP32 for the tensor-core objective epilogue
  float *w32;         // mu_cap: recombination weights in FP32 for the rank-mu staging
  void *Zm;           // kp x lam_cap, z in input format (candidate columns)
  float *Y32;         // kp x lam_cap, y = B D z from the FP32 accumulators
  double *fpart;      // ceil(n / 256) partial sums of the FP64 re-evaluation
  double fbest64;     // FP64 value of this generation's best point
  double *EX, *EG, *EH;  // ldn x n FP64 scratch of the refined eigensolver route (with EA, ET)
  float *jlog;        // FP32 Jacobi rotation log: jlog_steps_cap(n) x jlog_pairs(n) (c, s) pairs
  int *jlog_r;        // jlog_steps_cap(n): round-robin step index r of each logged step
  int jlog_steps, jlog_pad_;  // logged steps of the last FP32 Jacobi
  // many-CTA FP32 Jacobi (n > kEigMixedMaxN): two ring-layout buffers, two
  // P-long (c, s) record arrays, the last step that rotated, the step budget,
  // the rounding floor, and A32 = scale (A - shift I)
  float *jb_buf, *jb_rec;
  int jb_last_act, jb_tmax;
  float jb_floor;
  int jb_conv;           // converged: a whole-matrix check found nothing to rotate
  int jb_pend, jb_done;  // that check's pending flag and CTA count
  double jb_shift, jb_scale;
  int *err;           // device status word shared by the handle (kDevErr* bits)
  // tridiagonal route of the eigendecomposition (kernels_eig_trd.cu)
  int trd, trd_pad_;  // 1: this search's eigendecomposition takes the tridiagonal route
  double* trd_v;      // 11 x ldn doubles: d, e, split e, e^2, tau, eigenvalues (two orders), p and p.v buffers, scalars
  int* trd_i;         // 5 x ldn ints: block start / end, rank, cluster start, V^T V tile flags
  unsigned* trd_bar;  // the reduction's counters: group barrier, work per panel step (kTrdBarStride)
  unsigned char* ozp; // packed digit planes of the FP64-accurate tensor-core products (trd_oz_bytes)
  int* oze;           // their row exponents (trd_oz_exps ints)
};

// Flattened tiles of one kernel over a contiguous range of searches:
// tile t of the launch belongs to search s when off[s] <= t + off[s0] < off[s+1].
struct TileMap {
  const int* off;  // device, count + 1 prefix sums
  int s0, s1;      // search range [s0, s1)
  int total;       // off[s1] - off[s0]
};

// tile counts (host-side helpers, also used for prefix arrays)
__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
int tiles_sample_z(int n, int lam_cap);
int tiles_gemm_panel(int n, int lam_cap);   // 64 x 64 tiles of an n x lam panel
int tiles_colreduce(int lam_cap);
constexpr int kRankChunk = 1024;
int tiles_rank(int lam_cap);
int tiles_rank2d(int lam_cap);
int tiles_rows(int n);                      // 256-row blocks
int tiles_recomb(int n, int mu_cap);        // 32 rows x 256 ranks
int tiles_gemv(int n);                      // 32 rows x 256 columns
int part_doubles(int n, int ldn, int mu_cap);
int tiles_sym(int n);                       // upper 64 x 64 tiles of n x n
void cov_split(int n, int mu_cap, int* kc, int* nch);  // split of the rank-mu sum
int tiles_square(int n);                    // all 64 x 64 tiles of n x n

enum TileKind {
  TK_SAMPLE_Z = 0, TK_PANEL, TK_COLRED, TK_RANK, TK_ROWS, TK_RECOMB, TK_GEMV, TK_SYM, TK_SQUARE,
  TK_COVP, TK_RANK2D, TK_TCSAMPLE, TK_TCOBJ, TK_TCCOVP, TK_TCSYM, TK_FLAT, TK_FLATSYM, TK_REEVAL, TK_JBBLK, TK_JBLOAD, TK_JBROWS, TK_TRD, TK_TRDBIS, TK_TRDSQ, TK_TRDBT, TK_TRDOZP, TK_TRDOZG, TK_BTPACK, TK_BTGRAM, TK_BTTFAC, TK_BTROWS, TK_BTCOLS, TK_BTUPD, TK_BTFIN, TK_TRDS2KP, TK_TRDS2K, TK_COUNT
};

// launchers (kernels_gen.cu)
void launch_init_params(Search* S, int s0, int s1, DevOptions o, int reset_state, cudaStream_t st);
void launch_sample_z(Search* S, TileMap tm, DevOptions o, cudaStream_t st);
void launch_gemm_sample(Search* S, TileMap tm, cudaStream_t st);
void launch_gemm_objective(Search* S, TileMap tm, cudaStream_t st);
void launch_colreduce_f(Search* S, TileMap tm, cudaStream_t st);
void launch_rank(Search* S, TileMap tm2d, TileMap tm, cudaStream_t st);
void launch_recomb_partial(Search* S, TileMap tm, cudaStream_t st);
void launch_recomb_final(Search* S, TileMap tm, cudaStream_t st);
void launch_psigma_partial(Search* S, TileMap tm, cudaStream_t st);
void launch_psigma_final(Search* S, TileMap tm, cudaStream_t st);
void launch_finalize(Search* S, int s0, int s1, DevOptions o, cudaStream_t st);
void launch_cov_partial(Search* S, TileMap tm, cudaStream_t st);
void launch_cov_reduce(Search* S, TileMap tm, cudaStream_t st);
void launch_stop(Search* S, int s0, int s1, DevOptions o, cudaStream_t st);
void launch_force_restart(Search* S, int s, DevOptions o, cudaStream_t st);
// launchers (kernels_eig.cu)
void launch_eig_gemm_CB(Search* S, TileMap tm, cudaStream_t st);
void launch_eig_gemm_BtT(Search* S, TileMap tm, cudaStream_t st);
// Jacobi variants by dimension: one CTA per search with A and B in shared
// memory (n <= kJacobiSmallN), an 8-CTA cluster per search (kJacobiSmallN <
// n <= kJacobiClusterN), one CTA per search on global memory (larger n).
constexpr int kJacobiSmallN = 32;
constexpr int kJacobiClusterN = 256;
// Searches with kJacobiSmallN < n <= kEigBigMaxN (any precision) take the
// FP32-preconditioned, FP64-refined route of kernels_eig_mixed.cu: its FP32
// Jacobi runs in one CTA's shared memory up to kEigMixedMaxN
// (kernels_eig_mixed.cu) and as one launch per step over many CTAs above it
// (kernels_eig_big.cu). Larger n keep the plain warm-started FP64 Jacobi.
constexpr int kEigMixedMaxN = 160;
constexpr int kEigBigMaxN = 4096;
__host__ __device__ inline bool eig_refined_route(int n) { return n > kJacobiSmallN && n <= kEigBigMaxN; }
__host__ __device__ inline bool eig_refined_route(const Search& s) { return !s.trd && eig_refined_route(s.n); }
__host__ __device__ inline bool eig_big_route(int n) { return n > kEigMixedMaxN && n <= kEigBigMaxN; }
// The FP32 Jacobi of that route runs at most kJ32MaxSweeps sweeps of N - 1
// round-robin steps (N = n rounded up to even) in one CTA and logs the
// rotations of each step that rotates anything; the many-CTA form runs at
// most kJ32BigSweeps sweeps and logs every step. A logged step is N / 2
// (c, s) pairs, identity for idle pairs.
constexpr int kJ32MaxSweeps = 20;
constexpr int kJ32BigSweeps = 16;
__host__ __device__ inline int jlog_pairs(int n) { return (n + (n & 1)) / 2; }
__host__ __device__ inline int jlog_steps_cap(int n) {
  return (eig_big_route(n) ? kJ32BigSweeps : kJ32MaxSweeps) * (n + (n & 1) - 1);
}
void launch_jacobi_variant(Search* S, int s0, int s1, bool smem, int lo_n, int hi_n, int max_n,
                           cudaStream_t st);
void launch_jacobi_cluster(Search* S, int s0, int s1, int lo_n, int hi_n, int layout_n, cudaStream_t st);
void launch_set_bd(Search* S, TileMap tm, cudaStream_t st);
void launch_set_bd_force(Search* S, TileMap tm, cudaStream_t st);
int jacobi_smem_max_n();
int jacobi_smem_bytes(int n, bool smem_mats);

// mixed-precision path (kernels_mixed.cu)
int tiles_tc_sample(int n, int lam_cap);
int tiles_tc_objective(int lam_cap);
int tiles_tc_sym(int n);
void tc_cov_split(int n, int mu_cap, int* kc, int* nch);
int tc_elem_bytes(int precision);
void launch_tc_prepare_q(Search* S, int s, int precision, cudaStream_t st);
void launch_tc_set_bdt(Search* S, TileMap tm, int precision, int force, cudaStream_t st);
void launch_tc_set_bd_bdt(Search* S, TileMap tm, int precision, cudaStream_t st);  // BD and BDT together
void launch_tc_sample(Search* S, TileMap tm, int precision, cudaStream_t st);
void launch_tc_objective(Search* S, TileMap tm, int precision, cudaStream_t st);
void launch_tc_cov_partial(Search* S, TileMap tm, int precision, cudaStream_t st);
void launch_tc_cov_reduce(Search* S, TileMap tm, cudaStream_t st);
void launch_reeval(Search* S, TileMap tm, cudaStream_t st);
// mixed-precision eigensolver route (kernels_eig_mixed.cu): FP32 Jacobi
// sweeps, Newton-Schulz lift to FP64, then the FP64 Jacobi finishes
int tiles_flat(int n);
// 32-row blocks of the FP64 re-evaluation of the best point (one partial sum each)
__host__ __device__ inline int tiles_reeval(int n) { return (n + 31) / 32; }
int tiles_flat_sym(int n);
int launch_eig_mixed(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st);
// the refined route in two parts around the many-CTA FP32 Jacobi: the
// warm-start products (and the one-CTA FP32 Jacobi), then the refinement
int launch_eig_mixed_head(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st);
int launch_eig_mixed_tail(Search* S, TileMap tflat, TileMap tsym, int s0, int s1, int max_n, cudaStream_t st);
// launchers (kernels_eig_big.cu)
int tiles_jb_blocks(int n);
int tiles_jb_load(int n);
int tiles_jb_rows(int n);
size_t jb_buf_floats(int n);
void launch_j32b_start(Search* S, TileMap tload, int s0, int s1, cudaStream_t st);
void launch_j32b_step(Search* S, TileMap tblk, int t, cudaStream_t st);
void launch_j32b_check(Search* S, TileMap tblk, int t, cudaStream_t st);
void launch_jlog_big(Search* S, TileMap trows, int max_n, cudaStream_t st);

// Error text of calls that have no handle (read by cmaes_last_error(NULL)).
void set_global_error(const char* msg);

// tridiagonal route (kernels_eig_trd.cu): 32 < n <= kEigBigMaxN; the default
// above kEigAutoTrdN (below it the FP32 Jacobi of the refined route, in one
// CTA's shared memory, is faster)
constexpr int kEigAutoTrdN = kEigMixedMaxN;
constexpr int kTrdVectors = 11;  // Search::trd_v, in ldn doubles
constexpr int kTrdInts = 5;      // Search::trd_i, in ldn ints
int tiles_trd(int n);      // 128 eigenvalues per tile
int tiles_trd_bis(int n);  // 16 eigenvalues per tile (8 lanes each)
int tiles_trd_sq(int n);   // all 64 x 64 tiles of n x n
int tiles_trd_bt(int n);   // column groups of the back-transformation
int tiles_trd_ozp(int n);  // 64-row blocks of a packed n x n operand
int tiles_trd_ozg(int n);  // 128 x 64 tiles of the Gram matrix V^T V
size_t trd_oz_bytes(int n);  // Search::ozp
int trd_oz_exps(int n);      // Search::oze
// blocked back-transformation on the tensor cores (kernels_eig_trd_bt.cu)
int tiles_bt_pack(int n);    // 64-row blocks of every panel's Y^T and Y
int tiles_bt_gram(int n);    // two 128 x 64 tiles of Y^T Y per panel
int tiles_bt_tfac(int n);    // one per panel
int tiles_bt_rows(int n);    // 64-row blocks of a packed n-row operand
int tiles_bt_cols(int n);    // 64-column tiles of a 128 x n product
int tiles_bt_update(int n);  // 128 x 64 tiles of the largest panel's update
int tiles_bt_final(int n);   // 8 columns per tile
void bt_set_attributes();
size_t trd_reduce_smem(int max_n, int blocked);
int trd_reduce_blocks_per_sm(int max_n, int blocked);
int tiles_trd_s2k_pack(int n);  // 64-row blocks of the reduction's trailing-update operands
int tiles_trd_s2k(int n);       // 128 x 64 tiles of its trailing update
void trd_set_attributes(int max_n);
constexpr int kTrdStages = 6;  // reduction, eigenvalues, inverse iteration, clusters, orthogonalisation, back-transformation
constexpr int kTrdPanel = 64;  // columns per panel of the tridiagonal reduction
// counters per search of the reduction (Search::trd_bar): the group barrier,
// then one work counter per step of a panel
constexpr int kTrdBarStride = 1 + kTrdPanel;
// One cooperative launch of the reduction: CTAs [first, first + count) of the
// group table, all working on panel `panel` (-1: the unblocked form, the
// whole reduction in one launch).
struct TrdChunk {
  int first, count, panel;
};
struct TrdMaps {
  TileMap tt, tbis, tsq, tbt, ozp, ozg;  // TK_TRD, TK_TRDBIS, TK_TRDSQ, TK_TRDBT, TK_TRDOZP, TK_TRDOZG
  TileMap btpack, btgram, bttfac, btrows, btcols, btupd, btfin;  // TK_BTPACK .. TK_BTFIN
  TileMap s2kp, s2k;  // TK_TRDS2KP, TK_TRDS2K
};
int launch_bt(Search* S, const TrdMaps& m, int max_n, cudaStream_t st);
int launch_eig_trd(Search* S, const int4* grp, const TrdChunk* chunks, int nchunks, unsigned* bars,
                   int bar_count, int s0, int s1, const TrdMaps& tm, int max_n, int bis_lanes, cudaStream_t st,
                   cudaEvent_t* marks);

}  // namespace cmaes_gb300
