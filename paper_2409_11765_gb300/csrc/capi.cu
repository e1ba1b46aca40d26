// capi.cu -- the engine behind include/cmaes.h: device memory layout, the
// per-generation launch schedule, ask/tell, checkpoints and error handling.
//
// One handle holds `count` searches in one device arena. A generation is a
// fixed sequence of batched launches (sample, objective, rank + update,
// covariance, eigendecomposition when due, stop + restart), each covering all
// searches at once through prefix-summed tile lists; searches that are done or
// whose eigendecomposition is not due leave their tiles at once. All control
// decisions (restarts, lambda doubling, the lazy eigendecomposition cadence)
// are taken on the device, so the host only enqueues work, and a whole-batch
// generation replays one captured CUDA graph per phase.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cmaes.h"
#include "engine.h"

using namespace cmaes_gb300;

namespace {

struct PendingEvents {
  int first;  // index of the first of kNumPhases + 1 events in the pool
};

}  // namespace

struct cmaes_s {
  int count = 0;
  cmaes_options opt{};
  DevOptions dopt{};
  std::vector<Search> hs;  // host copies (constant fields authoritative)
  Search* dS = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int* d_off = nullptr;  // TK_COUNT x (count + 1)
  int* d_err = nullptr;  // device status word (bit 0: a bounded wait timed out)
  bool mixed = false;
  std::vector<int> h_off;
  cudaStream_t stream = nullptr;
  cmaes_status err = CMAES_OK;
  std::string msg;
  std::vector<int> ask_pending;
  int max_n = 0, max_n_small_jacobi = 0, max_n_cluster_jacobi = 0, max_n_global_jacobi = 0;
  bool any_rotated = false, any_sphere = false;
  bool any_plain_eig = false;  // a search outside the refined eigensolver route (warm start B^T C B by k_eig_gemm_*)
  int max_n_big = 0;           // largest n of the searches whose FP32 Jacobi runs over many CTAs
  // tridiagonal route: largest n, the CTA -> (search, member, group size) table
  // of the cooperative reduction, and one barrier counter per search
  int max_n_trd = 0;
  int trd_bis_lanes = 8;  // lanes per eigenvalue of the multisection (1 for large batches)
  int4* d_trd_grp = nullptr;
  int trd_grp_blocks = 0;
  std::vector<TrdChunk> trd_chunks;  // the cooperative launches of the reduction, panel by panel
  // per-stage times of the tridiagonal route in profiling mode: one set of
  // kTrdStages + 1 events per profiled generation, drained with the phases
  std::vector<cudaEvent_t> trd_pool;
  int trd_pending = 0;
  double trd_stage_ms[kTrdStages] = {0};
  cudaEvent_t* trd_marks = nullptr;  // events for the eigendecomposition being enqueued
  unsigned* d_trd_bar = nullptr;
  std::vector<Search> hs_probe;  // host copy of the searches, read between FP32 Jacobi sweeps
  long long launches = 0;
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> pool;
  std::vector<PendingEvents> pending;
  double phase_ms[kNumPhases] = {0};
  long long phase_launch[kNumPhases] = {0};
  // one CUDA graph per phase of a whole-batch generation, captured on first
  // use and replayed (the launch sequence of a handle is fixed: every control
  // decision is taken on the device); empty until then or after set_problem
  cudaGraphExec_t gexec[kNumPhases] = {nullptr};
  long long g_launch[kNumPhases] = {0};
  bool graphs_ready = false;

  TileMap tiles(int kind, int s0, int s1) const {
    TileMap tm;
    tm.off = d_off + static_cast<size_t>(kind) * (count + 1);
    tm.s0 = s0;
    tm.s1 = s1;
    const int* o = h_off.data() + static_cast<size_t>(kind) * (count + 1);
    tm.total = o[s1] - o[s0];
    return tm;
  }
};

static std::string g_create_error;

void cmaes_gb300::set_global_error(const char* msg) { g_create_error = msg; }

static cmaes_status set_error(cmaes_t h, cmaes_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) {
    h->msg = buf;
    if (st == CMAES_ECUDA) h->err = CMAES_ECUDA;
  } else {
    g_create_error = buf;
  }
  return st;
}

#define CUDA_TRY(h, call)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return set_error((h), CMAES_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

#define CHECK_HANDLE(h)                           \
  do {                                            \
    if (!(h)) return CMAES_EINVAL;                \
    if ((h)->err != CMAES_OK) return (h)->err;    \
  } while (0)

#define CHECK_SEARCH(h, s)                                                            \
  do {                                                                                \
    if ((s) < 0 || (s) >= (h)->count)                                                 \
      return set_error((h), CMAES_EINVAL, "search index %d out of range [0, %d)", (s), \
                       (h)->count);                                                   \
  } while (0)

static size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

static int default_lambda(int n) { return 4 + static_cast<int>(std::floor(3.0 * std::log(static_cast<double>(n)))); }

static cmaes_status launch_check(cmaes_t h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(h, CMAES_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return CMAES_OK;
}

// Reads the device status word (the handle's stream must be idle). A timed-out
// wait makes the handle unusable (sticky CMAES_ETIMEOUT); a non-finite state
// is reported once as CMAES_ENUMERIC and its bit cleared, since the stop test
// already restarted or ended the search.
static cmaes_status check_device_status(cmaes_t h) {
  int e = 0;
  CUDA_TRY(h, cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e & kDevErrTimeout) {
    h->err = CMAES_ETIMEOUT;
    h->msg = "a bounded device wait timed out";
    return CMAES_ETIMEOUT;
  }
  if (e & kDevErrNonFinite) {
    const int cleared = e & ~kDevErrNonFinite;
    CUDA_TRY(h, cudaMemcpy(h->d_err, &cleared, sizeof(int), cudaMemcpyHostToDevice));
    return set_error(h, CMAES_ENUMERIC, "a search's state became non-finite; the search was restarted or ended");
  }
  return CMAES_OK;
}

static cmaes_status read_search(cmaes_t h, int s, Search* out) {
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  cmaes_status r = check_device_status(h);
  if (r != CMAES_OK) return r;
  CUDA_TRY(h, cudaMemcpy(out, h->dS + s, sizeof(Search), cudaMemcpyDeviceToHost));
  return CMAES_OK;
}

static cmaes_status write_search(cmaes_t h, int s, const Search* in) {
  CUDA_TRY(h, cudaMemcpy(h->dS + s, in, sizeof(Search), cudaMemcpyHostToDevice));
  return CMAES_OK;
}

// ------------------------------ phase schedule ------------------------------
// Counts the launches each launcher actually issues (grids of zero are not
// launched).
static inline void count_launch(cmaes_t h, int phase, int total) {
  if (total > 0) {
    h->launches += 1;
    h->phase_launch[phase] += 1;
  }
}

static void enqueue_sample(cmaes_t h, int s0, int s1, cudaStream_t st) {
  TileMap a = h->tiles(TK_SAMPLE_Z, s0, s1);
  launch_sample_z(h->dS, a, h->dopt, st);
  count_launch(h, kPhaseSample, a.total);
  if (h->mixed) {
    TileMap b = h->tiles(TK_TCSAMPLE, s0, s1);
    launch_tc_sample(h->dS, b, h->opt.precision, st);
    count_launch(h, kPhaseSample, b.total);
  } else {
    TileMap b = h->tiles(TK_PANEL, s0, s1);
    launch_gemm_sample(h->dS, b, st);
    count_launch(h, kPhaseSample, b.total);
  }
}

static void enqueue_objective(cmaes_t h, int s0, int s1, cudaStream_t st) {
  TileMap b = h->tiles(TK_COLRED, s0, s1);
  if (h->any_rotated) {
    if (h->mixed) {
      TileMap a = h->tiles(TK_TCOBJ, s0, s1);
      launch_tc_objective(h->dS, a, h->opt.precision, st);
      count_launch(h, kPhaseObjective, a.total);
    } else {
      TileMap a = h->tiles(TK_PANEL, s0, s1);
      launch_gemm_objective(h->dS, a, st);
      count_launch(h, kPhaseObjective, a.total);
    }
  }
  if (!h->mixed || h->any_sphere) {
    launch_colreduce_f(h->dS, b, st);
    count_launch(h, kPhaseObjective, b.total);
  }
}

static void enqueue_update(cmaes_t h, int s0, int s1, cudaStream_t st) {
  TileMap r = h->tiles(TK_RANK, s0, s1), rc = h->tiles(TK_RECOMB, s0, s1);
  TileMap r2 = h->tiles(TK_RANK2D, s0, s1);
  TileMap rows = h->tiles(TK_ROWS, s0, s1), gv = h->tiles(TK_GEMV, s0, s1);
  launch_rank(h->dS, r2, r, st);
  count_launch(h, kPhaseUpdate, r2.total);
  count_launch(h, kPhaseUpdate, r.total);
  if (h->mixed) {
    TileMap re = h->tiles(TK_REEVAL, s0, s1);
    launch_reeval(h->dS, re, st);
    count_launch(h, kPhaseUpdate, re.total);
  }
  launch_recomb_partial(h->dS, rc, st);
  count_launch(h, kPhaseUpdate, rc.total);
  launch_recomb_final(h->dS, rows, st);
  count_launch(h, kPhaseUpdate, rows.total);
  launch_psigma_partial(h->dS, gv, st);
  count_launch(h, kPhaseUpdate, gv.total);
  launch_psigma_final(h->dS, rows, st);
  count_launch(h, kPhaseUpdate, rows.total);
  launch_finalize(h->dS, s0, s1, h->dopt, st);
  count_launch(h, kPhaseUpdate, s1 - s0);
}

static void enqueue_cov(cmaes_t h, int s0, int s1, cudaStream_t st) {
  if (h->mixed) {
    TileMap p = h->tiles(TK_TCCOVP, s0, s1), t = h->tiles(TK_TCSYM, s0, s1);
    launch_tc_cov_partial(h->dS, p, h->opt.precision, st);
    count_launch(h, kPhaseCov, p.total);
    launch_tc_cov_reduce(h->dS, t, st);
    count_launch(h, kPhaseCov, t.total);
    return;
  }
  TileMap p = h->tiles(TK_COVP, s0, s1), t = h->tiles(TK_SYM, s0, s1);
  launch_cov_partial(h->dS, p, st);
  count_launch(h, kPhaseCov, p.total);
  launch_cov_reduce(h->dS, t, st);
  count_launch(h, kPhaseCov, t.total);
}

// The many-CTA FP32 Jacobi of the refined route (n > kEigMixedMaxN): one
// launch per step over the large searches of [s0, s1). Once per sweep of the
// largest of them the host reads the searches back and stops when each has
// converged (a full quiet window after its last rotation) or spent its
// budget. Needs the stream to be synchronisable: this phase is never captured
// in a graph while such searches exist.
static int enqueue_jacobi32_big(cmaes_t h, int s0, int s1, cudaStream_t st) {
  TileMap tload = h->tiles(TK_JBLOAD, s0, s1), tblk = h->tiles(TK_JBBLK, s0, s1);
  TileMap trows = h->tiles(TK_JBROWS, s0, s1);
  if (tblk.total <= 0) return 0;
  int nl = 3;
  launch_j32b_start(h->dS, tload, s0, s1, st);
  int Mmax = 0;
  for (int s = s0; s < s1; ++s) {
    const int n = h->hs[s].n;
    if (eig_big_route(n)) Mmax = std::max(Mmax, n + (n & 1) - 1);
  }
  const int tcap = kJ32BigSweeps * Mmax;
  h->hs_probe.resize(h->count);
  for (int t = 0; t < tcap; ++t) {
    if (t > 0 && t % 64 == 0) {  // ends the quiet window early once nothing is left to rotate
      launch_j32b_check(h->dS, tblk, t, st);
      ++nl;
    }
    launch_j32b_step(h->dS, tblk, t, st);
    ++nl;
    if ((t + 1) % Mmax == 0 && t + 1 < tcap) {
      if (cudaMemcpyAsync(h->hs_probe.data() + s0, h->dS + s0, sizeof(Search) * (s1 - s0), cudaMemcpyDeviceToHost,
                          st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        break;  // the sticky error surfaces at the next check
      bool running = false;
      for (int s = s0; s < s1 && !running; ++s) {
        const Search& x = h->hs_probe[s];
        if (x.done || !x.eig_due || !eig_big_route(x.n)) continue;
        const int M = x.n + (x.n & 1) - 1;
        running = !x.jb_conv && (t + 1 < x.jb_tmax) && (t + 1 - x.jb_last_act < M);
      }
      if (!running) break;
    }
  }
  launch_jlog_big(h->dS, trows, h->max_n_big, st);
  return nl + 1;
}

static void enqueue_eig(cmaes_t h, int s0, int s1, cudaStream_t st) {
  TileMap sq = h->tiles(TK_SQUARE, s0, s1);
  if (h->max_n_trd > 0) {
    // the cooperative reduction always covers every search of the handle (its
    // group table is fixed at create); the searches outside [s0, s1) that
    // are due are reduced too, which only repeats their decomposition
    const TrdMaps tmaps{h->tiles(TK_TRD, s0, s1),   h->tiles(TK_TRDBIS, s0, s1), h->tiles(TK_TRDSQ, s0, s1),
                        h->tiles(TK_TRDBT, s0, s1), h->tiles(TK_TRDOZP, s0, s1), h->tiles(TK_TRDOZG, s0, s1),
                        h->tiles(TK_BTPACK, s0, s1), h->tiles(TK_BTGRAM, s0, s1), h->tiles(TK_BTTFAC, s0, s1),
                        h->tiles(TK_BTROWS, s0, s1), h->tiles(TK_BTCOLS, s0, s1), h->tiles(TK_BTUPD, s0, s1),
                        h->tiles(TK_BTFIN, s0, s1),  h->tiles(TK_TRDS2KP, s0, s1), h->tiles(TK_TRDS2K, s0, s1)};
    const int nl = launch_eig_trd(h->dS, h->d_trd_grp, h->trd_chunks.data(), static_cast<int>(h->trd_chunks.size()),
                                  h->d_trd_bar, h->count, s0, s1, tmaps, h->max_n_trd, h->trd_bis_lanes, st,
                                  h->trd_marks);
    h->launches += nl;
    h->phase_launch[kPhaseEig] += nl;
  }
  {
    TileMap tfl = h->tiles(TK_FLAT, s0, s1);
    TileMap tsy = h->tiles(TK_FLATSYM, s0, s1);
    int nl = launch_eig_mixed_head(h->dS, tfl, tsy, s0, s1, h->max_n, st);
    if (h->max_n_big > 0) nl += enqueue_jacobi32_big(h, s0, s1, st);
    nl += launch_eig_mixed_tail(h->dS, tfl, tsy, s0, s1, h->max_n, st);
    h->launches += nl;
    h->phase_launch[kPhaseEig] += nl;
  }
  if (h->any_plain_eig) {
    launch_eig_gemm_CB(h->dS, sq, st);
    count_launch(h, kPhaseEig, sq.total);
    launch_eig_gemm_BtT(h->dS, sq, st);
    count_launch(h, kPhaseEig, sq.total);
  }
  if (h->max_n_small_jacobi > 0) {
    launch_jacobi_variant(h->dS, s0, s1, true, 0, kJacobiSmallN, h->max_n_small_jacobi, st);
    count_launch(h, kPhaseEig, s1 - s0);
  }
  if (h->max_n_cluster_jacobi > 0) {
    launch_jacobi_cluster(h->dS, s0, s1, kJacobiSmallN, kJacobiClusterN, h->max_n_cluster_jacobi, st);
    count_launch(h, kPhaseEig, s1 - s0);
  }
  if (h->max_n_global_jacobi > 0) {
    launch_jacobi_variant(h->dS, s0, s1, false, kJacobiClusterN, 1 << 30, h->max_n_global_jacobi, st);
    count_launch(h, kPhaseEig, s1 - s0);
  }
  if (h->mixed) {
    launch_tc_set_bd_bdt(h->dS, sq, h->opt.precision, st);  // B diag(D) in FP64 and in the operand format
    count_launch(h, kPhaseEig, sq.total);
  } else {
    launch_set_bd(h->dS, sq, st);
    count_launch(h, kPhaseEig, sq.total);
  }
}

static void enqueue_stop(cmaes_t h, int s0, int s1, cudaStream_t st) {
  launch_stop(h->dS, s0, s1, h->dopt, st);
  count_launch(h, kPhaseStop, s1 - s0);
}

static cmaes_status record_event(cmaes_t h, int idx, cudaStream_t st) {
  CUDA_TRY(h, cudaEventRecord(h->pool[idx], st));
  return CMAES_OK;
}

static cmaes_status drain_trd_events(cmaes_t h) {
  if (h->trd_pending == 0) return CMAES_OK;
  const int need = kTrdStages + 1;
  CUDA_TRY(h, cudaEventSynchronize(h->trd_pool[h->trd_pending * need - 1]));
  for (int p = 0; p < h->trd_pending; ++p)
    for (int k = 0; k < kTrdStages; ++k) {
      float ms = 0.f;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, h->trd_pool[p * need + k], h->trd_pool[p * need + k + 1]));
      h->trd_stage_ms[k] += ms;
    }
  h->trd_pending = 0;
  return CMAES_OK;
}

static cmaes_status drain_events(cmaes_t h) {
  cmaes_status rt = drain_trd_events(h);
  if (rt != CMAES_OK) return rt;
  if (h->pending.empty()) return CMAES_OK;
  CUDA_TRY(h, cudaEventSynchronize(h->pool[h->pending.back().first + kNumPhases]));
  for (const PendingEvents& p : h->pending) {
    for (int k = 0; k < kNumPhases; ++k) {
      float ms = 0.f;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, h->pool[p.first + k], h->pool[p.first + k + 1]));
      h->phase_ms[k] += ms;
    }
  }
  h->pending.clear();
  return CMAES_OK;
}

static void enqueue_phase(cmaes_t h, int k, int s0, int s1, cudaStream_t st) {
  switch (k) {
    case kPhaseSample: enqueue_sample(h, s0, s1, st); break;
    case kPhaseObjective: enqueue_objective(h, s0, s1, st); break;
    case kPhaseUpdate: enqueue_update(h, s0, s1, st); break;
    case kPhaseCov: enqueue_cov(h, s0, s1, st); break;
    case kPhaseEig: enqueue_eig(h, s0, s1, st); break;
    default: enqueue_stop(h, s0, s1, st); break;
  }
}

static void drop_graphs(cmaes_t h) {
  for (int k = 0; k < kNumPhases; ++k) {
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    h->gexec[k] = nullptr;
    h->g_launch[k] = 0;
  }
  h->graphs_ready = false;
}

// Captures each phase of a whole-batch generation into a graph on the handle's
// stream (nothing runs during capture; the launch counters are restored).
static cmaes_status ensure_graphs(cmaes_t h) {
  if (h->graphs_ready) return CMAES_OK;
  for (int k = 0; k < kNumPhases; ++k) {
    if (k == kPhaseEig && h->max_n_big > 0) continue;  // host-driven: enqueued directly
    const long long l0 = h->launches, p0 = h->phase_launch[k];
    cudaGraph_t g = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
    enqueue_phase(h, k, 0, h->count, h->stream);
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    const long long nl = h->launches - l0;
    h->launches = l0;
    h->phase_launch[k] = p0;
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      drop_graphs(h);
      return set_error(h, CMAES_ECUDA, "capture of phase %d failed: %s", k, cudaGetErrorString(e));
    }
    cudaError_t ei = cudaSuccess;
    if (nl > 0) ei = cudaGraphInstantiate(&h->gexec[k], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      drop_graphs(h);
      return set_error(h, CMAES_ECUDA, "graph of phase %d: %s", k, cudaGetErrorString(ei));
    }
    h->g_launch[k] = nl;
  }
  h->graphs_ready = true;
  return launch_check(h, "graph capture");
}

static cmaes_status enqueue_generation(cmaes_t h, int s0, int s1, cudaStream_t st, bool with_objective) {
  const bool prof = h->profiling;
  const bool graphed = (s0 == 0 && s1 == h->count);
  if (graphed) {
    cmaes_status rg = ensure_graphs(h);
    if (rg != CMAES_OK) return rg;
  }
  auto run = [&](int k) -> cmaes_status {
    if (k == kPhaseEig && prof && h->max_n_trd > 0) {
      // profiling: enqueued directly, with events between the stages of the
      // tridiagonal route
      const int need = kTrdStages + 1;
      if (h->trd_pending >= 256) {
        cmaes_status rd = drain_trd_events(h);
        if (rd != CMAES_OK) return rd;
      }
      while (static_cast<int>(h->trd_pool.size()) < (h->trd_pending + 1) * need) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreate(&e));
        h->trd_pool.push_back(e);
      }
      h->trd_marks = h->trd_pool.data() + h->trd_pending * need;
      enqueue_phase(h, k, s0, s1, st);
      h->trd_marks = nullptr;
      ++h->trd_pending;
      return CMAES_OK;
    }
    if (!graphed || (k == kPhaseEig && h->max_n_big > 0)) {
      enqueue_phase(h, k, s0, s1, st);
      return CMAES_OK;
    }
    if (h->gexec[k]) {
      CUDA_TRY(h, cudaGraphLaunch(h->gexec[k], st));
      h->launches += h->g_launch[k];
      h->phase_launch[k] += h->g_launch[k];
    }
    return CMAES_OK;
  };
  int base = 0;
  if (prof) {
    const int need = kNumPhases + 1;
    if (static_cast<int>(h->pool.size()) < static_cast<int>(h->pending.size() + 1) * need) {
      if (h->pool.size() >= 4096) {
        cmaes_status r = drain_events(h);
        if (r != CMAES_OK) return r;
      }
      while (static_cast<int>(h->pool.size()) < static_cast<int>(h->pending.size() + 1) * need) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreate(&e));
        h->pool.push_back(e);
      }
    }
    base = static_cast<int>(h->pending.size()) * need;
    h->pending.push_back({base});
  }
  auto mark = [&](int k) -> cmaes_status {
    return prof ? record_event(h, base + k, st) : CMAES_OK;
  };
  cmaes_status r;
  for (int k = 0; k < kNumPhases; ++k) {
    if ((r = mark(k)) != CMAES_OK) return r;
    if (with_objective || (k != kPhaseSample && k != kPhaseObjective))
      if ((r = run(k)) != CMAES_OK) return r;
  }
  if ((r = mark(kNumPhases)) != CMAES_OK) return r;
  return launch_check(h, "generation");
}

// ---------------------------------- ABI -------------------------------------
extern "C" {

void cmaes_default_options(cmaes_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CMAES_FP64;
  o->max_restarts = 0;
  o->ipop_double = 1;
  o->eig_every = 0;
  o->max_iter = 0;
  o->stop_mask = CMAES_STOP_ALL;
  o->f_target = -INFINITY;
  o->box_lo = -4.0;
  o->box_hi = 4.0;
  o->tol_hist_fun = 1e-12;
  o->tol_x_factor = 1e-12;
  o->cond_max = 1e14;
}

const char* cmaes_strerror(cmaes_status st) {
  switch (st) {
    case CMAES_OK: return "ok";
    case CMAES_EINVAL: return "invalid argument";
    case CMAES_ENOMEM: return "out of memory";
    case CMAES_ECUDA: return "CUDA error";
    case CMAES_ESTATE: return "call out of order";
    case CMAES_ETIMEOUT: return "device wait timed out";
    case CMAES_ENUMERIC: return "non-finite state";
    case CMAES_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* cmaes_last_error(cmaes_t h) { return h ? h->msg.c_str() : g_create_error.c_str(); }

void cmaes_destroy(cmaes_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  if (h->arena) cudaFree(h->arena);
  if (h->dS) cudaFree(h->dS);
  if (h->d_off) cudaFree(h->d_off);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_trd_grp) cudaFree(h->d_trd_grp);
  for (cudaEvent_t e : h->trd_pool) cudaEventDestroy(e);
  if (h->d_trd_bar) cudaFree(h->d_trd_bar);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

cmaes_status cmaes_create_batch(int count, const int* n_arr, const int* lam_arr, const double* const* x0,
                                const double* sigma0, uint64_t seed, const cmaes_options* opt_in,
                                cmaes_t* out) {
  if (!out) return set_error(nullptr, CMAES_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !n_arr || !x0 || !sigma0)
    return set_error(nullptr, CMAES_EINVAL, "count must be >= 1 and n, x0, sigma0 non-NULL");
  if (count > (1 << 24)) return set_error(nullptr, CMAES_EINVAL, "at most 2^24 searches");
  cmaes_options opt;
  if (opt_in) opt = *opt_in; else cmaes_default_options(&opt);
  if (opt.precision < CMAES_FP64 || opt.precision > CMAES_MIXED_BF16)
    return set_error(nullptr, CMAES_EINVAL, "unknown precision %d", opt.precision);
  if (opt.max_restarts < 0 || opt.max_restarts > 255)
    return set_error(nullptr, CMAES_EINVAL, "max_restarts must be in [0, 255]");
  if (!(opt.box_lo < opt.box_hi)) return set_error(nullptr, CMAES_EINVAL, "box_lo must be < box_hi");
  if (opt.eig_method < CMAES_EIG_AUTO || opt.eig_method > CMAES_EIG_TRIDIAGONAL)
    return set_error(nullptr, CMAES_EINVAL, "unknown eig_method %d", opt.eig_method);

  cmaes_t h = new cmaes_s();
  h->count = count;
  h->opt = opt;
  h->mixed = opt.precision != CMAES_FP64;
  const int esz = tc_elem_bytes(opt.precision);
  DevOptions& d = h->dopt;
  d.max_restarts = opt.max_restarts;
  d.ipop_double = opt.ipop_double ? 1 : 0;
  d.eig_every = opt.eig_every;
  d.max_iter = opt.max_iter;
  d.stop_mask = opt.stop_mask;
  d.precision = opt.precision;
  d.restart_hold = opt.restart_hold ? 1 : 0;
  d.f_target = opt.f_target;
  d.box_lo = opt.box_lo;
  d.box_hi = opt.box_hi;
  d.tol_hist_fun = opt.tol_hist_fun;
  d.tol_x_factor = opt.tol_x_factor;
  d.cond_max = opt.cond_max;
  d.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFu);
  d.key1 = static_cast<uint32_t>(seed >> 32);

  // layout
  h->hs.resize(count);
  size_t total = 0;
  std::vector<size_t> base(count);
  for (int s = 0; s < count; ++s) {
    const int n = n_arr[s];
    int lam = lam_arr ? lam_arr[s] : 0;
    if (n < 1 || n > 65536) { delete h; return set_error(nullptr, CMAES_EINVAL, "search %d: n=%d out of range", s, n); }
    if (lam == 0) lam = default_lambda(n);
    if (lam < 2) { delete h; return set_error(nullptr, CMAES_EINVAL, "search %d: lambda=%d < 2", s, lam); }
    if (!(sigma0[s] > 0.0) || !x0[s]) { delete h; return set_error(nullptr, CMAES_EINVAL, "search %d: bad sigma0 or x0", s); }
    long long cap = opt.ipop_double ? (static_cast<long long>(lam) << opt.max_restarts) : lam;
    if (cap > (1LL << 24)) { delete h; return set_error(nullptr, CMAES_EINVAL, "search %d: lambda capacity %lld too large", s, cap); }
    Search& x = h->hs[s];
    std::memset(&x, 0, sizeof(x));
    x.n = n;
    x.ldn = (n + 15) & ~15;
    x.lam0 = lam;
    x.lam_cap = static_cast<int>(cap);
    x.mu_cap = x.lam_cap / 2;
    x.hist_cap = 10 + static_cast<int>(std::ceil(30.0 * n / lam));
    x.index = s;
    x.obj = 0;
    x.sigma0 = sigma0[s];
    cov_split(n, x.mu_cap, &x.cov_kc, &x.cov_nch);
    x.mixed = h->mixed ? opt.precision : 0;
    x.kp = (n + 31) & ~31;
    x.trd = (eig_refined_route(n) &&
             (opt.eig_method == CMAES_EIG_TRIDIAGONAL || (opt.eig_method == CMAES_EIG_AUTO && n > kEigAutoTrdN)))
                ? 1 : 0;
    if (h->mixed) tc_cov_split(n, x.mu_cap, &x.covm_kc, &x.covm_nch);
    const size_t ldn = x.ldn, n_ = n, lc = x.lam_cap, kp = x.kp;
    size_t b = 0;
    b += 9 * align256(ldn * 8);                       // vectors
    b += align256(static_cast<size_t>(x.mu_cap) * 8);  // w
    b += align256(static_cast<size_t>(2 * x.hist_cap) * 8);  // best f, then its mixed-evaluation error
    b += align256(static_cast<size_t>(part_doubles(n, x.ldn, x.mu_cap)) * 8);
    if (h->mixed) {
      b += align256(static_cast<size_t>(tiles_tc_sym(n)) * x.covm_nch * 16384 * 8);
      b += 3 * align256(n_ * kp * esz);                // BDT QTh QTl
      b += align256(kp * lc * esz) + align256(kp * lc * 4);  // Zm Y32
      b += align256(static_cast<size_t>(tiles_reeval(n)) * 8);
      b += align256(n_ * 4);                             // lam32
      b += align256(static_cast<size_t>(x.mu_cap) * 4);  // w32
      b += align256(ldn * lc * 8);                     // X
    } else {
      if (x.cov_nch > 1) b += align256(static_cast<size_t>(tiles_sym(n)) * x.cov_nch * 4096 * 8);
      b += 4 * align256(ldn * lc * 8);                 // Z Y X U
    }
    b += 6 * align256(ldn * n_ * 8);                   // C B BD Q EA ET
    if (eig_refined_route(n)) b += 3 * align256(ldn * n_ * 8);  // EX EG EH
    if (eig_refined_route(n) && !x.trd) {
      b += align256(static_cast<size_t>(jlog_steps_cap(n)) * jlog_pairs(n) * 8);  // jlog
      b += align256(static_cast<size_t>(jlog_steps_cap(n)) * 4);                  // jlog_r
    }
    if (x.trd)
      b += align256(ldn * kTrdVectors * 8) + align256(ldn * kTrdInts * 4) + align256(trd_oz_bytes(n)) +
           align256(static_cast<size_t>(trd_oz_exps(n)) * 4);
    if (eig_big_route(n) && !x.trd) {
      b += align256(jb_buf_floats(n) * 4);                         // jb_buf
      b += align256(static_cast<size_t>(jlog_pairs(n)) * 16);      // jb_rec
    }
    b += align256(lc * 8);                             // f
    b += 2 * align256(lc * 4);                         // order rank
    base[s] = total;
    total += b;
    if (n > h->max_n) h->max_n = n;
    if (!eig_refined_route(n)) h->any_plain_eig = true;
    if (x.trd) {
      if (n > h->max_n_trd) h->max_n_trd = n;
    } else {
      if (eig_big_route(n) && n > h->max_n_big) h->max_n_big = n;
      int* jm = n <= kJacobiSmallN ? &h->max_n_small_jacobi
                : n <= kJacobiClusterN ? &h->max_n_cluster_jacobi : &h->max_n_global_jacobi;
      if (n > *jm) *jm = n;
    }
  }
  h->arena_bytes = total;
  cudaError_t e = cudaMalloc(&h->arena, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return set_error(nullptr, CMAES_ENOMEM, "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
  }
  auto fail = [&](cmaes_status st) {
    g_create_error = h->msg;
    cmaes_destroy(h);
    return st;
  };
#define CREATE_TRY(call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      set_error(h, CMAES_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                \
      return fail(CMAES_ECUDA);                                                                  \
    }                                                                                            \
  } while (0)
  CREATE_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  CREATE_TRY(cudaMemsetAsync(h->arena, 0, total, h->stream));
  for (int s = 0; s < count; ++s) {
    Search& x = h->hs[s];
    char* p = h->arena + base[s];
    const size_t ldn = x.ldn, n_ = x.n, lc = x.lam_cap;
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    x.m = reinterpret_cast<double*>(take(ldn * 8));
    x.ps = reinterpret_cast<double*>(take(ldn * 8));
    x.pc = reinterpret_cast<double*>(take(ldn * 8));
    x.D = reinterpret_cast<double*>(take(ldn * 8));
    x.xstar = reinterpret_cast<double*>(take(ldn * 8));
    x.lamdiag = reinterpret_cast<double*>(take(ldn * 8));
    x.best_x = reinterpret_cast<double*>(take(ldn * 8));
    x.yw = reinterpret_cast<double*>(take(ldn * 8));
    x.zw = reinterpret_cast<double*>(take(ldn * 8));
    x.w = reinterpret_cast<double*>(take(static_cast<size_t>(x.mu_cap) * 8));
    x.hist = reinterpret_cast<double*>(take(static_cast<size_t>(2 * x.hist_cap) * 8));
    x.part = reinterpret_cast<double*>(take(static_cast<size_t>(part_doubles(x.n, x.ldn, x.mu_cap)) * 8));
    const size_t kp = x.kp;
    if (h->mixed) {
      x.covpart = reinterpret_cast<double*>(take(static_cast<size_t>(tiles_tc_sym(x.n)) * x.covm_nch * 16384 * 8));
      x.BDT = take(n_ * kp * esz);
      x.QTh = take(n_ * kp * esz);
      x.QTl = take(n_ * kp * esz);
      x.Zm = take(kp * lc * esz);
      x.Y32 = reinterpret_cast<float*>(take(kp * lc * 4));
      x.fpart = reinterpret_cast<double*>(take(static_cast<size_t>(tiles_reeval(x.n)) * 8));
      x.lam32 = reinterpret_cast<float*>(take(n_ * 4));
      x.w32 = reinterpret_cast<float*>(take(static_cast<size_t>(x.mu_cap) * 4));
    } else {
      x.covpart = x.cov_nch > 1
                      ? reinterpret_cast<double*>(take(static_cast<size_t>(tiles_sym(x.n)) * x.cov_nch * 4096 * 8))
                      : nullptr;
    }
    x.C = reinterpret_cast<double*>(take(ldn * n_ * 8));
    x.B = reinterpret_cast<double*>(take(ldn * n_ * 8));
    x.BD = reinterpret_cast<double*>(take(ldn * n_ * 8));
    x.Q = reinterpret_cast<double*>(take(ldn * n_ * 8));
    x.EA = reinterpret_cast<double*>(take(ldn * n_ * 8));
    x.ET = reinterpret_cast<double*>(take(ldn * n_ * 8));
    if (eig_refined_route(x.n)) {
      x.EX = reinterpret_cast<double*>(take(ldn * n_ * 8));
      x.EG = reinterpret_cast<double*>(take(ldn * n_ * 8));
      x.EH = reinterpret_cast<double*>(take(ldn * n_ * 8));
    }
    if (eig_refined_route(x.n) && !x.trd) {
      x.jlog = reinterpret_cast<float*>(take(static_cast<size_t>(jlog_steps_cap(x.n)) * jlog_pairs(x.n) * 8));
      x.jlog_r = reinterpret_cast<int*>(take(static_cast<size_t>(jlog_steps_cap(x.n)) * 4));
    }
    if (x.trd) {
      x.trd_v = reinterpret_cast<double*>(take(ldn * kTrdVectors * 8));
      x.trd_i = reinterpret_cast<int*>(take(ldn * kTrdInts * 4));
      x.ozp = reinterpret_cast<unsigned char*>(take(trd_oz_bytes(x.n)));
      x.oze = reinterpret_cast<int*>(take(static_cast<size_t>(trd_oz_exps(x.n)) * 4));
    }
    if (eig_big_route(x.n) && !x.trd) {
      x.jb_buf = reinterpret_cast<float*>(take(jb_buf_floats(x.n) * 4));
      x.jb_rec = reinterpret_cast<float*>(take(static_cast<size_t>(jlog_pairs(x.n)) * 16));
    }
    if (h->mixed) {
      x.X = reinterpret_cast<double*>(take(ldn * lc * 8));
    } else {
      x.Z = reinterpret_cast<double*>(take(ldn * lc * 8));
      x.Y = reinterpret_cast<double*>(take(ldn * lc * 8));
      x.X = reinterpret_cast<double*>(take(ldn * lc * 8));
      x.U = reinterpret_cast<double*>(take(ldn * lc * 8));
    }
    x.f = reinterpret_cast<double*>(take(lc * 8));
    x.order = reinterpret_cast<int*>(take(lc * 4));
    x.rank = reinterpret_cast<int*>(take(lc * 4));
    CREATE_TRY(cudaMemcpyAsync(x.m, x0[s], n_ * 8, cudaMemcpyHostToDevice, h->stream));
  }
  CREATE_TRY(cudaMalloc(&h->d_err, sizeof(int)));
  CREATE_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  for (int s = 0; s < count; ++s) h->hs[s].err = h->d_err;
  if (h->max_n_trd > 0) {
    CREATE_TRY(cudaMalloc(&h->d_trd_bar, sizeof(unsigned) * count * kTrdBarStride));
    CREATE_TRY(cudaMemsetAsync(h->d_trd_bar, 0, sizeof(unsigned) * count * kTrdBarStride, h->stream));
    for (int s = 0; s < count; ++s)
      if (h->hs[s].trd) h->hs[s].trd_bar = h->d_trd_bar + static_cast<size_t>(s) * kTrdBarStride;
    // groups of the cooperative reduction, within what can be resident at once
    int dev = 0, sms = 0;
    CREATE_TRY(cudaGetDevice(&dev));
    CREATE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    trd_set_attributes(h->max_n_trd);
    // the largest group of a search: at least 16 columns per CTA, and enough
    // work per step to outweigh the group barriers ((n - 64 q)^2 / 16384)
    auto gcap = [](long long m) { return std::max(1, static_cast<int>(std::min(m / 16, m * m / 16384))); };
    // the unblocked form (one barrier per step) when every search can have its
    // largest group at once: the GPU is then partly idle and a step's latency
    // sets the time; the panel form otherwise
    long long caps = 0;
    for (int s = 0; s < count; ++s)
      if (h->hs[s].trd) caps += gcap(h->hs[s].n);
    const long long budget_u = static_cast<long long>(trd_reduce_blocks_per_sm(h->max_n_trd, 0)) * sms;
    const bool blocked = caps > budget_u;
    const int per_sm = trd_reduce_blocks_per_sm(h->max_n_trd, blocked ? 1 : 0);
    long long budget = static_cast<long long>(per_sm) * sms;
    if (budget < 1) {
      set_error(h, CMAES_EUNSUPPORTED, "the tridiagonal reduction cannot be resident on this device");
      return fail(CMAES_EUNSUPPORTED);
    }
    // the panel form: one group table per panel of kTrdPanel columns: the searches with
    // columns left in panel q share the resident CTAs in proportion to their
    // trailing work (n - kTrdPanel q)^2, each with at least one CTA and at most
    // (n - kTrdPanel q) / 16 and (n - kTrdPanel q)^2 / 16384 (enough work per
    // step to outweigh the group barriers); launches of at most `budget` CTAs
    // never split a group
    std::vector<int4> grp;
    h->trd_chunks.clear();
    if (!blocked) {
      for (int s = 0; s < count; ++s) {
        if (!h->hs[s].trd) continue;
        const int G = gcap(h->hs[s].n);
        for (int r = 0; r < G; ++r) grp.push_back(make_int4(s, r, G, 0));
      }
      h->trd_chunks.push_back(TrdChunk{0, static_cast<int>(grp.size()), -1});
    }
    const int panels = blocked ? ceil_div(h->max_n_trd, kTrdPanel) : 0;
    for (int q = 0; q < panels; ++q) {
      double wsum = 0.0;
      int nact = 0;
      for (int s = 0; s < count; ++s) {
        const Search& x = h->hs[s];
        if (!x.trd || x.n <= kTrdPanel * q) continue;
        const double m = static_cast<double>(x.n - kTrdPanel * q);
        wsum += m * m;
        ++nact;
      }
      if (nact == 0) continue;
      const long long spare = budget > nact ? budget - nact : 0;
      int chunk_start = static_cast<int>(grp.size());
      for (int s = 0; s < count; ++s) {
        const Search& x = h->hs[s];
        if (!x.trd || x.n <= kTrdPanel * q) continue;
        const long long m = x.n - kTrdPanel * q;
        const double share = static_cast<double>(m * m) / wsum;
        int G = static_cast<int>(std::floor(share * static_cast<double>(spare))) + 1;
        G = std::min(G, gcap(m));
        if (static_cast<long long>(grp.size()) + G - chunk_start > budget) {
          h->trd_chunks.push_back(TrdChunk{chunk_start, static_cast<int>(grp.size()) - chunk_start, q});
          chunk_start = static_cast<int>(grp.size());
        }
        for (int r = 0; r < G; ++r) grp.push_back(make_int4(s, r, G, 0));
      }
      h->trd_chunks.push_back(TrdChunk{chunk_start, static_cast<int>(grp.size()) - chunk_start, q});
    }
    h->trd_grp_blocks = static_cast<int>(grp.size());
    // eigenvalues to find per decomposition of the whole batch: with more than
    // the GPU holds as 8-lane groups, plain bisection does the least work
    long long eig_total = 0;
    for (int s = 0; s < count; ++s)
      if (h->hs[s].trd) eig_total += h->hs[s].n;
    h->trd_bis_lanes = eig_total * 8 > static_cast<long long>(sms) * 2048 ? 1 : 8;
    CREATE_TRY(cudaMalloc(&h->d_trd_grp, sizeof(int4) * grp.size()));
    CREATE_TRY(cudaMemcpyAsync(h->d_trd_grp, grp.data(), sizeof(int4) * grp.size(), cudaMemcpyHostToDevice,
                               h->stream));
    CREATE_TRY(cudaStreamSynchronize(h->stream));  // grp (host vector) leaves scope
  }
  CREATE_TRY(cudaMalloc(&h->dS, sizeof(Search) * count));
  CREATE_TRY(cudaMemcpyAsync(h->dS, h->hs.data(), sizeof(Search) * count, cudaMemcpyHostToDevice, h->stream));
  // tile prefix sums per kind
  h->h_off.assign(static_cast<size_t>(TK_COUNT) * (count + 1), 0);
  for (int k = 0; k < TK_COUNT; ++k) {
    int* o = h->h_off.data() + static_cast<size_t>(k) * (count + 1);
    long long acc = 0;
    for (int s = 0; s < count; ++s) {
      const Search& x = h->hs[s];
      int t = 0;
      switch (k) {
        case TK_SAMPLE_Z: t = tiles_sample_z(x.n, x.lam_cap); break;
        case TK_PANEL: t = tiles_gemm_panel(x.n, x.lam_cap); break;
        case TK_COLRED: t = tiles_colreduce(x.lam_cap); break;
        case TK_RANK: t = tiles_rank(x.lam_cap); break;
        case TK_ROWS: t = tiles_rows(x.n); break;
        case TK_RECOMB: t = tiles_recomb(x.n, x.mu_cap); break;
        case TK_GEMV: t = tiles_gemv(x.n); break;
        case TK_SYM: t = 4 * tiles_sym(x.n); break;  // reduce: 4 blocks per tile
        case TK_SQUARE: t = tiles_square(x.n); break;
        case TK_COVP: t = tiles_sym(x.n) * x.cov_nch; break;
        case TK_RANK2D: t = tiles_rank2d(x.lam_cap); break;
        case TK_TCSAMPLE: t = h->mixed ? tiles_tc_sample(x.n, x.lam_cap) : 0; break;
        case TK_TCOBJ: t = h->mixed ? tiles_tc_objective(x.lam_cap) : 0; break;
        case TK_TCCOVP: t = h->mixed ? tiles_tc_sym(x.n) * x.covm_nch : 0; break;
        case TK_TCSYM: t = h->mixed ? 16 * tiles_tc_sym(x.n) : 0; break;  // reduce: 16 blocks per tile
        case TK_FLAT: t = eig_refined_route(x) ? tiles_flat(x.n) : 0; break;
        case TK_REEVAL: t = h->mixed ? tiles_reeval(x.n) : 0; break;
        case TK_FLATSYM: t = eig_refined_route(x) ? tiles_flat_sym(x.n) : 0; break;
        case TK_TRD: t = x.trd ? tiles_trd(x.n) : 0; break;
        case TK_TRDBIS: t = x.trd ? tiles_trd_bis(x.n) : 0; break;
        case TK_TRDSQ: t = x.trd ? tiles_trd_sq(x.n) : 0; break;
        case TK_TRDBT: t = x.trd ? tiles_trd_bt(x.n) : 0; break;
        case TK_TRDOZP: t = x.trd ? tiles_trd_ozp(x.n) : 0; break;
        case TK_TRDOZG: t = x.trd ? tiles_trd_ozg(x.n) : 0; break;
        case TK_BTPACK: t = x.trd ? tiles_bt_pack(x.n) : 0; break;
        case TK_BTGRAM: t = x.trd ? tiles_bt_gram(x.n) : 0; break;
        case TK_BTTFAC: t = x.trd ? tiles_bt_tfac(x.n) : 0; break;
        case TK_BTROWS: t = x.trd ? tiles_bt_rows(x.n) : 0; break;
        case TK_BTCOLS: t = x.trd ? tiles_bt_cols(x.n) : 0; break;
        case TK_BTUPD: t = x.trd ? tiles_bt_update(x.n) : 0; break;
        case TK_BTFIN: t = x.trd ? tiles_bt_final(x.n) : 0; break;
        case TK_TRDS2KP: t = x.trd ? tiles_trd_s2k_pack(x.n) : 0; break;
        case TK_TRDS2K: t = x.trd ? tiles_trd_s2k(x.n) : 0; break;
        case TK_JBBLK: t = x.trd ? 0 : tiles_jb_blocks(x.n); break;
        case TK_JBLOAD: t = x.trd ? 0 : tiles_jb_load(x.n); break;
        case TK_JBROWS: t = x.trd ? 0 : tiles_jb_rows(x.n); break;
      }
      o[s] = static_cast<int>(acc);
      acc += t;
    }
    if (acc > 0x7fffffff) {
      set_error(h, CMAES_EINVAL, "tile count overflow");
      return fail(CMAES_EINVAL);
    }
    o[count] = static_cast<int>(acc);
  }
  CREATE_TRY(cudaMalloc(&h->d_off, sizeof(int) * h->h_off.size()));
  CREATE_TRY(cudaMemcpyAsync(h->d_off, h->h_off.data(), sizeof(int) * h->h_off.size(), cudaMemcpyHostToDevice,
                             h->stream));
  launch_init_params(h->dS, 0, count, h->dopt, 1, h->stream);
  h->launches += 1;
  if (h->mixed) {  // B D = I in the tensor-core format
    launch_tc_set_bdt(h->dS, h->tiles(TK_SQUARE, 0, count), opt.precision, 1, h->stream);
    h->launches += 1;
  }
  CREATE_TRY(cudaGetLastError());
  CREATE_TRY(cudaStreamSynchronize(h->stream));
  h->ask_pending.assign(count, 0);
  *out = h;
  return CMAES_OK;
#undef CREATE_TRY
}

cmaes_status cmaes_create(int n, int lambda, const double* x0, double sigma0, uint64_t seed,
                          const cmaes_options* opt, cmaes_t* out) {
  const double* xs[1] = {x0};
  return cmaes_create_batch(1, &n, &lambda, xs, &sigma0, seed, opt, out);
}

int cmaes_count(cmaes_t h) { return h ? h->count : 0; }

cmaes_status cmaes_set_problem(cmaes_t h, int s, int kind, const double* Q, const double* lambda_diag,
                               const double* xstar) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (kind < CMAES_OBJ_ELLIPSOID || kind > CMAES_OBJ_SPHERE)
    return set_error(h, CMAES_EINVAL, "unknown objective kind %d", kind);
  if (!xstar) return set_error(h, CMAES_EINVAL, "xstar is NULL");
  if (kind != CMAES_OBJ_SPHERE && !Q) return set_error(h, CMAES_EINVAL, "Q is NULL");
  if (kind == CMAES_OBJ_ELLIPSOID && !lambda_diag) return set_error(h, CMAES_EINVAL, "lambda_diag is NULL");
  Search& x = h->hs[s];
  const size_t n = x.n, ldn = x.ldn;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(x.xstar, xstar, n * 8, cudaMemcpyHostToDevice));
  if (Q) CUDA_TRY(h, cudaMemcpy2D(x.Q, ldn * 8, Q, n * 8, n * 8, n, cudaMemcpyHostToDevice));
  if (lambda_diag) CUDA_TRY(h, cudaMemcpy(x.lamdiag, lambda_diag, n * 8, cudaMemcpyHostToDevice));
  x.obj = kind;
  CUDA_TRY(h, cudaMemcpy(&h->dS[s].obj, &x.obj, sizeof(int), cudaMemcpyHostToDevice));
  if (h->mixed && kind != CMAES_OBJ_SPHERE) {
    launch_tc_prepare_q(h->dS, s, h->opt.precision, h->stream);
    h->launches += 1;
    cmaes_status r = launch_check(h, "prepare_q");
    if (r != CMAES_OK) return r;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  drop_graphs(h);  // the objective phase's launches depend on the objective kinds
  h->any_rotated = false;
  h->any_sphere = false;
  for (const Search& y : h->hs) {
    if (y.obj == CMAES_OBJ_ELLIPSOID || y.obj == CMAES_OBJ_RASTRIGIN) h->any_rotated = true;
    if (y.obj == CMAES_OBJ_SPHERE) h->any_sphere = true;
  }
  return CMAES_OK;
}

cmaes_status cmaes_step_batch(cmaes_t h, int generations, void* stream) {
  CHECK_HANDLE(h);
  if (generations < 0) return set_error(h, CMAES_EINVAL, "generations < 0");
  for (int s = 0; s < h->count; ++s) {
    if (h->hs[s].obj == CMAES_OBJ_NONE) return set_error(h, CMAES_EINVAL, "search %d has no objective", s);
    if (h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d has an ask pending", s);
  }
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  if (st != h->stream) {
    // order this call after earlier work on the handle's own stream
    cudaEvent_t ev;
    CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(h, cudaEventRecord(ev, h->stream));
    CUDA_TRY(h, cudaStreamWaitEvent(st, ev, 0));
    CUDA_TRY(h, cudaEventDestroy(ev));
  }
  for (int g = 0; g < generations; ++g) {
    cmaes_status r = enqueue_generation(h, 0, h->count, st, true);
    if (r != CMAES_OK) return r;
  }
  if (st != h->stream) {
    cudaEvent_t ev;
    CUDA_TRY(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(h, cudaEventRecord(ev, st));
    CUDA_TRY(h, cudaStreamWaitEvent(h->stream, ev, 0));
    CUDA_TRY(h, cudaEventDestroy(ev));
  }
  return CMAES_OK;
}

cmaes_status cmaes_inject_status(cmaes_t h, int bits) {
  CHECK_HANDLE(h);
  if (bits & ~(kDevErrTimeout | kDevErrNonFinite))
    return set_error(h, CMAES_EINVAL, "unknown status bits 0x%x", bits);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int e = 0;
  CUDA_TRY(h, cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  e |= bits;
  CUDA_TRY(h, cudaMemcpy(h->d_err, &e, sizeof(int), cudaMemcpyHostToDevice));
  return CMAES_OK;
}

cmaes_status cmaes_sync(cmaes_t h) {
  CHECK_HANDLE(h);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_status(h);
}

cmaes_status cmaes_ask_device(cmaes_t h, int s, const double** X_dev, int* ld) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: ask pending, call tell first", s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  if (cur.done) return set_error(h, CMAES_ESTATE, "search %d is done", s);
  enqueue_sample(h, s, s + 1, h->stream);
  if ((r = launch_check(h, "sample")) != CMAES_OK) return r;
  h->ask_pending[s] = 1;
  if (X_dev) *X_dev = h->hs[s].X;
  if (ld) *ld = h->hs[s].ldn;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return CMAES_OK;
}

cmaes_status cmaes_ask(cmaes_t h, int s, double* X_host) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (!X_host) return set_error(h, CMAES_EINVAL, "X_host is NULL");
  cmaes_status r = cmaes_ask_device(h, s, nullptr, nullptr);
  if (r != CMAES_OK) return r;
  Search cur;
  if ((r = read_search(h, s, &cur)) != CMAES_OK) return r;
  const Search& x = h->hs[s];
  CUDA_TRY(h, cudaMemcpy2D(X_host, static_cast<size_t>(x.n) * 8, x.X, static_cast<size_t>(x.ldn) * 8,
                           static_cast<size_t>(x.n) * 8, cur.lam, cudaMemcpyDeviceToHost));
  return CMAES_OK;
}

cmaes_status cmaes_tell(cmaes_t h, int s, const double* f_host) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (!f_host) return set_error(h, CMAES_EINVAL, "f_host is NULL");
  if (!h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: tell without ask", s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  CUDA_TRY(h, cudaMemcpy(h->hs[s].f, f_host, static_cast<size_t>(cur.lam) * 8, cudaMemcpyHostToDevice));
  if ((r = enqueue_generation(h, s, s + 1, h->stream, false)) != CMAES_OK) return r;
  h->ask_pending[s] = 0;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return CMAES_OK;
}

static cmaes_status check_range(cmaes_t h, int s0, int s1) {
  if (s0 < 0 || s1 > h->count || s0 >= s1)
    return set_error(h, CMAES_EINVAL, "search range [%d, %d) outside [0, %d)", s0, s1, h->count);
  return CMAES_OK;
}

cmaes_status cmaes_ask_async(cmaes_t h, int s0, int s1, double* const* X, int* lam_done, void* stream) {
  CHECK_HANDLE(h);
  cmaes_status r = check_range(h, s0, s1);
  if (r != CMAES_OK) return r;
  if (!X || !lam_done) return set_error(h, CMAES_EINVAL, "X or lam_done is NULL");
  for (int s = s0; s < s1; ++s) {
    if (!X[s - s0]) return set_error(h, CMAES_EINVAL, "X[%d] is NULL", s - s0);
    if (h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: ask pending, call tell first", s);
  }
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  enqueue_sample(h, s0, s1, st);
  for (int s = s0; s < s1; ++s) {
    const Search& x = h->hs[s];
    CUDA_TRY(h, cudaMemcpy2DAsync(X[s - s0], static_cast<size_t>(x.n) * 8, x.X, static_cast<size_t>(x.ldn) * 8,
                                  static_cast<size_t>(x.n) * 8, x.lam_cap, cudaMemcpyDeviceToHost, st));
    const char* dev = reinterpret_cast<const char*>(h->dS + s);
    CUDA_TRY(h, cudaMemcpyAsync(lam_done + 2 * (s - s0), dev + offsetof(Search, lam), sizeof(int),
                                cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaMemcpyAsync(lam_done + 2 * (s - s0) + 1, dev + offsetof(Search, done), sizeof(int),
                                cudaMemcpyDeviceToHost, st));
    h->ask_pending[s] = 1;
  }
  return launch_check(h, "ask_async");
}

cmaes_status cmaes_tell_async(cmaes_t h, int s0, int s1, const double* const* f, void* stream) {
  CHECK_HANDLE(h);
  cmaes_status r = check_range(h, s0, s1);
  if (r != CMAES_OK) return r;
  if (!f) return set_error(h, CMAES_EINVAL, "f is NULL");
  for (int s = s0; s < s1; ++s) {
    if (!f[s - s0]) return set_error(h, CMAES_EINVAL, "f[%d] is NULL", s - s0);
    if (!h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: tell without ask", s);
  }
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
  for (int s = s0; s < s1; ++s)
    CUDA_TRY(h, cudaMemcpyAsync(h->hs[s].f, f[s - s0], static_cast<size_t>(h->hs[s].lam_cap) * 8,
                                cudaMemcpyHostToDevice, st));
  if ((r = enqueue_generation(h, s0, s1, st, false)) != CMAES_OK) return r;
  for (int s = s0; s < s1; ++s) h->ask_pending[s] = 0;
  return CMAES_OK;
}

cmaes_status cmaes_restart(cmaes_t h, int s) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: ask pending", s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  if (cur.done == 1) return set_error(h, CMAES_ESTATE, "search %d is done", s);
  if (h->dopt.ipop_double && static_cast<long long>(cur.lam) * 2 > h->hs[s].lam_cap)
    return set_error(h, CMAES_ESTATE, "search %d: restart budget exhausted", s);
  launch_force_restart(h->dS, s, h->dopt, h->stream);
  h->launches += 1;
  if ((r = launch_check(h, "restart")) != CMAES_OK) return r;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return CMAES_OK;
}

cmaes_status cmaes_best(cmaes_t h, int s, double* x, double* f) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  if (f) *f = cur.best_f;
  if (x) CUDA_TRY(h, cudaMemcpy(x, h->hs[s].best_x, static_cast<size_t>(cur.n) * 8, cudaMemcpyDeviceToHost));
  return CMAES_OK;
}

cmaes_status cmaes_query(cmaes_t h, int s, int* lambda, int* gen, int* restart, int* flags, int* done) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  if (lambda) *lambda = cur.lam;
  if (gen) *gen = cur.gen;
  if (restart) *restart = cur.restart;
  if (flags) *flags = cur.flags;
  if (done) *done = cur.done;
  return CMAES_OK;
}

cmaes_status cmaes_get_generation(cmaes_t h, int s, double* X, double* f, int* order) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  const Search& x = h->hs[s];
  const size_t n = x.n, lam = cur.lam;
  if (X) CUDA_TRY(h, cudaMemcpy2D(X, n * 8, x.X, static_cast<size_t>(x.ldn) * 8, n * 8, lam, cudaMemcpyDeviceToHost));
  if (f) CUDA_TRY(h, cudaMemcpy(f, x.f, lam * 8, cudaMemcpyDeviceToHost));
  if (order) CUDA_TRY(h, cudaMemcpy(order, x.order, lam * 4, cudaMemcpyDeviceToHost));
  return CMAES_OK;
}

cmaes_status cmaes_get_state(cmaes_t h, int s, cmaes_state* st) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (!st) return set_error(h, CMAES_EINVAL, "state is NULL");
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  const Search& x = h->hs[s];
  const size_t n = x.n, ldn = x.ldn;
  st->n = x.n;
  st->lambda = cur.lam;
  st->gen = cur.gen;
  st->restart = cur.restart;
  st->done = cur.done;
  st->flags = cur.flags;
  st->sigma = cur.sigma;
  st->best_f = cur.best_f;
  const int cnt = cur.hist_count < cur.hist_len ? cur.hist_count : cur.hist_len;
  st->hist_count = cnt;
  if (st->m) CUDA_TRY(h, cudaMemcpy(st->m, x.m, n * 8, cudaMemcpyDeviceToHost));
  if (st->ps) CUDA_TRY(h, cudaMemcpy(st->ps, x.ps, n * 8, cudaMemcpyDeviceToHost));
  if (st->pc) CUDA_TRY(h, cudaMemcpy(st->pc, x.pc, n * 8, cudaMemcpyDeviceToHost));
  if (st->D) CUDA_TRY(h, cudaMemcpy(st->D, x.D, n * 8, cudaMemcpyDeviceToHost));
  if (st->best_x) CUDA_TRY(h, cudaMemcpy(st->best_x, x.best_x, n * 8, cudaMemcpyDeviceToHost));
  if (st->C) CUDA_TRY(h, cudaMemcpy2D(st->C, n * 8, x.C, ldn * 8, n * 8, n, cudaMemcpyDeviceToHost));
  if (st->B) CUDA_TRY(h, cudaMemcpy2D(st->B, n * 8, x.B, ldn * 8, n * 8, n, cudaMemcpyDeviceToHost));
  if (st->hist && cnt > 0) {
    std::vector<double> ring(cur.hist_len);
    CUDA_TRY(h, cudaMemcpy(ring.data(), x.hist, static_cast<size_t>(cur.hist_len) * 8, cudaMemcpyDeviceToHost));
    const int start = cur.hist_count <= cur.hist_len ? 0 : cur.hist_count % cur.hist_len;
    for (int q = 0; q < cnt; ++q) st->hist[q] = ring[(start + q) % cur.hist_len];
  }
  return CMAES_OK;
}

cmaes_status cmaes_set_state(cmaes_t h, int s, const cmaes_state* st) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  if (!st) return set_error(h, CMAES_EINVAL, "state is NULL");
  const Search& x = h->hs[s];
  if (st->n != x.n) return set_error(h, CMAES_EINVAL, "state n=%d does not match search n=%d", st->n, x.n);
  if (st->lambda < x.lam0 || st->lambda > x.lam_cap)
    return set_error(h, CMAES_EINVAL, "lambda=%d outside [%d, %d]", st->lambda, x.lam0, x.lam_cap);
  if (h->ask_pending[s]) return set_error(h, CMAES_ESTATE, "search %d: ask pending", s);
  // a non-finite sigma is accepted like a non-finite m (a checkpoint of a
  // broken state): the next generation's stop test restarts or ends the search
  if (st->gen < 0 || st->restart < 0 || st->restart > 255 || (std::isfinite(st->sigma) && !(st->sigma > 0.0)))
    return set_error(h, CMAES_EINVAL, "bad gen, restart or sigma");
  const int hist_len = 10 + static_cast<int>(std::ceil(30.0 * x.n / st->lambda));
  if (st->hist_count < 0 || (st->hist_count > 0 && !st->hist))
    return set_error(h, CMAES_EINVAL, "bad hist");
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  const size_t n = x.n, ldn = x.ldn;
  cur.lam = st->lambda;
  cur.gen = st->gen;
  cur.restart = st->restart;
  cur.done = st->done;
  cur.flags = st->flags;
  cur.sigma = st->sigma;
  cur.best_f = st->best_f;
  cur.eig_due = 0;
  const int keep = st->hist_count < hist_len ? st->hist_count : hist_len;
  cur.hist_count = keep;
  // the snapshot holds no evaluation errors: a restored window counts them as 0
  CUDA_TRY(h, cudaMemset(x.hist + x.hist_cap, 0, static_cast<size_t>(x.hist_cap) * 8));
  if (keep > 0) {
    CUDA_TRY(h, cudaMemcpy(x.hist, st->hist + (st->hist_count - keep), static_cast<size_t>(keep) * 8,
                           cudaMemcpyHostToDevice));
  }
  if ((r = write_search(h, s, &cur)) != CMAES_OK) return r;
  if (st->m) CUDA_TRY(h, cudaMemcpy(x.m, st->m, n * 8, cudaMemcpyHostToDevice));
  if (st->ps) CUDA_TRY(h, cudaMemcpy(x.ps, st->ps, n * 8, cudaMemcpyHostToDevice));
  if (st->pc) CUDA_TRY(h, cudaMemcpy(x.pc, st->pc, n * 8, cudaMemcpyHostToDevice));
  if (st->D) CUDA_TRY(h, cudaMemcpy(x.D, st->D, n * 8, cudaMemcpyHostToDevice));
  if (st->best_x) CUDA_TRY(h, cudaMemcpy(x.best_x, st->best_x, n * 8, cudaMemcpyHostToDevice));
  if (st->C) CUDA_TRY(h, cudaMemcpy2D(x.C, ldn * 8, st->C, n * 8, n * 8, n, cudaMemcpyHostToDevice));
  if (st->B) CUDA_TRY(h, cudaMemcpy2D(x.B, ldn * 8, st->B, n * 8, n * 8, n, cudaMemcpyHostToDevice));
  launch_init_params(h->dS, s, s + 1, h->dopt, 0, h->stream);
  h->launches += 1;
  TileMap sq = h->tiles(TK_SQUARE, s, s + 1);
  launch_set_bd_force(h->dS, sq, h->stream);
  h->launches += 1;
  if (h->mixed) {
    launch_tc_set_bdt(h->dS, sq, h->opt.precision, 1, h->stream);
    h->launches += 1;
  }
  if ((r = launch_check(h, "set_state")) != CMAES_OK) return r;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return CMAES_OK;
}

cmaes_status cmaes_set_profiling(cmaes_t h, int enable) {
  CHECK_HANDLE(h);
  if (!enable) {
    cmaes_status r = drain_events(h);
    if (r != CMAES_OK) return r;
  }
  h->profiling = enable != 0;
  return CMAES_OK;
}

cmaes_status cmaes_phase_times(cmaes_t h, double* ms, long long* launches, int reset) {
  CHECK_HANDLE(h);
  cmaes_status r = drain_events(h);
  if (r != CMAES_OK) return r;
  for (int k = 0; k < kNumPhases; ++k) {
    if (ms) ms[k] = h->phase_ms[k];
    if (launches) launches[k] = h->phase_launch[k];
  }
  if (reset) {
    for (int k = 0; k < kNumPhases; ++k) {
      h->phase_ms[k] = 0.0;
      h->phase_launch[k] = 0;
    }
  }
  return CMAES_OK;
}

cmaes_status cmaes_eig_stage_times(cmaes_t h, double* ms, int reset) {
  CHECK_HANDLE(h);
  cmaes_status r = drain_events(h);
  if (r != CMAES_OK) return r;
  for (int k = 0; k < kTrdStages; ++k) {
    if (ms) ms[k] = h->trd_stage_ms[k];
    if (reset) h->trd_stage_ms[k] = 0.0;
  }
  return CMAES_OK;
}

cmaes_status cmaes_eig_stats(cmaes_t h, int s, long long* decompositions, long long* sweeps,
                             long long* rotations, long long* sweeps32) {
  CHECK_HANDLE(h);
  CHECK_SEARCH(h, s);
  Search cur;
  cmaes_status r = read_search(h, s, &cur);
  if (r != CMAES_OK) return r;
  if (decompositions) *decompositions = cur.eig_count;
  if (sweeps) *sweeps = cur.eig_sweeps_total;
  if (rotations) *rotations = cur.eig_rotations;
  if (sweeps32) *sweeps32 = cur.eig_sweeps32;
  return CMAES_OK;
}

long long cmaes_kernel_launches(cmaes_t h) { return h ? h->launches : 0; }

}  // extern "C"
