/*
 * cmaes.h -- C ABI of the GB300 batched IPOP-CMA-ES engine.
 *
 * The engine runs many independent CMA-ES searches ("descents") on one GPU.
 * Each generation of each search performs, on the device:
 *   - sampling of lambda points x_k = m + sigma B D z_k, z_k ~ N(0, I)
 *     (paper §2.1, Eq. (1); all k at once as the GEMM of §3.1),
 *   - evaluation of a built-in objective, or of caller-supplied values
 *     (Algorithm 1, lines 7-9; the objective is a black box, §1),
 *   - the update of (m, C, sigma, p_sigma, p_c) from the ranked points
 *     (Algorithm 1, line 10; Eq. (2), rewritten as Eq. (3) in §3.1),
 *   - the eigendecomposition C = B D^2 B^T, every g_eig generations (§2.1),
 *   - the stop tests of §2.2 and the IPOP restart of Algorithm 2 (lambda
 *     doubled at each restart) or, with ipop_double = 0, a restart at the same
 *     lambda (the concurrent K-Distributed layout of §3.2.3).
 *
 * Conventions (all entry points):
 *   - Every call returns a cmaes_status; none throws, aborts or exits.
 *   - A CUDA error is sticky: once a call returns CMAES_ECUDA, every later call
 *     on that handle returns CMAES_ECUDA (cmaes_last_error() gives the text).
 *     So is a device wait that gave up: every device wait (tensor-core
 *     mbarriers) is bounded, and one that runs out records it in the handle's
 *     device status word; the next call that reads that word (cmaes_sync and
 *     every call that synchronises) and every later call return
 *     CMAES_ETIMEOUT.
 *   - NaN / infinite objective values are accepted and ranked last. When a
 *     search's state itself becomes non-finite (m, sigma or diag C), its stop
 *     test (CMAES_STOP_NONFINITE) restarts or ends that search, and the next
 *     call that reads the device status word returns CMAES_ENUMERIC once; the
 *     handle stays usable.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership. Host arrays passed out are caller-allocated and sized as
 *     documented. Matrices are n x n, column-major, leading dimension n.
 *   - Population panels are n x lambda, column-major (one candidate per column,
 *     leading dimension n).
 *   - A handle is not thread-safe; calls on one handle must be serialised.
 *   - The engine owns all of its device memory (allocated in cmaes_create*,
 *     released in cmaes_destroy).
 */
#ifndef CMAES_GB300_CMAES_H
#define CMAES_GB300_CMAES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmaes_s* cmaes_t;

typedef enum {
    CMAES_OK = 0,
    CMAES_EINVAL = 1,      /* bad argument (size, index, null pointer, option) */
    CMAES_ENOMEM = 2,      /* device or host allocation failed */
    CMAES_ECUDA = 3,       /* a CUDA call failed; the handle is poisoned */
    CMAES_ESTATE = 4,      /* call out of order (tell without ask, search done) */
    CMAES_ETIMEOUT = 5,    /* a bounded device wait gave up */
    CMAES_ENUMERIC = 6,    /* the search state became non-finite */
    CMAES_EUNSUPPORTED = 7 /* valid request this build does not provide */
} cmaes_status;

/* Arithmetic of the sampling, objective and rank-mu GEMMs. The eigensolver,
 * the mean, the paths and sigma are FP64 in every mode. */
typedef enum {
    CMAES_FP64 = 0,
    CMAES_MIXED_TF32 = 1,
    CMAES_MIXED_BF16 = 2
} cmaes_precision;

/* Built-in synthetic objectives (stand-ins for the BBOB families of §4.1):
 *   ELLIPSOID  f = sum_i Lambda_i u_i^2,               u = Q (x - x*)
 *   RASTRIGIN  f = 10 n + sum_i (u_i^2 - 10 cos(2 pi u_i))
 *   SPHERE     f = sum_i (x_i - x*_i)^2                                    */
typedef enum {
    CMAES_OBJ_NONE = 0,
    CMAES_OBJ_ELLIPSOID = 1,
    CMAES_OBJ_RASTRIGIN = 2,
    CMAES_OBJ_SPHERE = 3
} cmaes_objective;

/* Stop criteria (§2.2: quality not improving, locally flat, distribution too
 * small; constants after Auger & Hansen 2005). Bit mask. */
#define CMAES_STOP_FTARGET 1        /* best f < f_target: the search ends      */
#define CMAES_STOP_MAXITER 2        /* generations >= max_iter                 */
#define CMAES_STOP_TOLHISTFUN 4     /* range of recent best f < tol_hist_fun   */
                                    /* (mixed handles: or < 10 x the largest   */
                                    /* |f_mixed - f_FP64| of those best points) */
#define CMAES_STOP_TOLX 8           /* sigma * max(|p_c|, sqrt(diag C)) < tolx */
#define CMAES_STOP_CONDITIONCOV 16  /* cond(C) > cond_max                      */
#define CMAES_STOP_NOEFFECTAXIS 32  /* 0.1 sigma D_j b_j does not move m       */
#define CMAES_STOP_NOEFFECTCOORD 64 /* 0.2 sigma sqrt(C_ii) does not move m_i  */
#define CMAES_STOP_NONFINITE 128    /* m, sigma or diag C not finite           */
#define CMAES_STOP_ALL 255

/* Eigensolver of C = B D^2 B^T for 32 < n <= 4096 (smaller n always use a
 * one-CTA FP64 Jacobi; larger n a warm-started FP64 Jacobi on one CTA).
 *   JACOBI: warm-started from the previous basis; cyclic Jacobi sweeps in
 *     FP32, FP64 accuracy recovered by two Ogita-Aishima refinement steps
 *     and a Newton-Schulz step, then an FP64 Jacobi cleanup.
 *   TRIDIAGONAL: Householder reduction to tridiagonal form, the route of
 *     LAPACK's dsyev that the paper calls (§3.1): bisection for the
 *     eigenvalues, inverse iteration for the eigenvectors, Newton-Schulz
 *     steps for orthogonality, all in FP64.
 *   AUTO (default): JACOBI up to n = 160 (its FP32 sweeps fit one CTA's
 *     shared memory and beat the reduction's n sequential FP64 steps there),
 *     TRIDIAGONAL above (the Jacobi sweeps' n steps each then span the GPU). */
typedef enum {
    CMAES_EIG_AUTO = 0,
    CMAES_EIG_JACOBI = 1,
    CMAES_EIG_TRIDIAGONAL = 2
} cmaes_eig_method;

typedef struct cmaes_options {
    int precision;        /* cmaes_precision                                  */
    int max_restarts;     /* descents after the first; K_max = 2^max_restarts */
    int ipop_double;      /* 1: lambda <- 2 lambda per restart (Algorithm 2)   */
    int eig_every;        /* 0: lazy rule max(1, floor(1/((c1+cmu) n 10)))     */
    int max_iter;         /* 0: 100 + 50 (n+3)^2 / sqrt(lambda)                */
    int stop_mask;        /* CMAES_STOP_* bits that may fire                   */
    double f_target;      /* -inf disables                                     */
    double box_lo;        /* search box of the restart means (§4.1)            */
    double box_hi;
    double tol_hist_fun;  /* default 1e-12                                     */
    double tol_x_factor;  /* TolX = tol_x_factor * sigma0, default 1e-12       */
    double cond_max;      /* default 1e14                                      */
    int restart_hold;     /* 0: a stopped descent restarts on the device       */
                          /* (Algorithm 2). 1: it pauses (cmaes_query reports   */
                          /* done = 2) until cmaes_restart resumes it, so the   */
                          /* host can schedule descents (K-Replicated, §3.2.2)  */
    int eig_method;       /* cmaes_eig_method: eigensolver for 32 < n <= 4096   */
} cmaes_options;

/* Snapshot of one search (checkpoint / resume, and teacher-forced checks).
 * Pointer members are caller-owned host arrays; NULL skips that member.
 * cmaes_get_state fills them; cmaes_set_state reads them (and recomputes the
 * lambda-dependent strategy constants on the device). */
typedef struct cmaes_state {
    int n;            /* dimension (read-only: checked on set)                 */
    int lambda;       /* current population size                               */
    int gen;          /* generations done in the current descent               */
    int restart;      /* descent number (0 = first)                            */
    int done;         /* 1 when the search has ended                           */
    int flags;        /* stop flags of the last generation                     */
    int hist_count;   /* entries in hist (most recent last)                    */
    double sigma;
    double best_f;    /* best f over all descents                              */
    double* m;        /* n                                                     */
    double* ps;       /* n: p_sigma                                            */
    double* pc;       /* n: p_c                                                */
    double* D;        /* n: square roots of the eigenvalues of C               */
    double* best_x;   /* n                                                     */
    double* C;        /* n*n                                                   */
    double* B;        /* n*n: orthonormal eigenvectors of C (columns)          */
    double* hist;     /* capacity 10 + ceil(30 n / lambda0) entries            */
} cmaes_state;

/* Fills *opt with the defaults listed above (FP64, no restarts, lazy eig). */
void cmaes_default_options(cmaes_options* opt);

/* One search. n >= 1; lambda >= 2 (0 selects 4 + floor(3 ln n)); x0: host, n
 * doubles, the first mean; sigma0 > 0; seed keys the Philox4x32-10 streams of
 * all draws (z, restart means). opt may be NULL (defaults). Errors: EINVAL,
 * ENOMEM, ECUDA. On error *out is NULL. */
cmaes_status cmaes_create(int n, int lambda, const double* x0, double sigma0,
                          uint64_t seed, const cmaes_options* opt, cmaes_t* out);

/* count searches of uneven (n, lambda) in one handle. n, lambda, sigma0: host
 * arrays of count entries; x0: host array of count pointers to n[s] doubles.
 * Search s draws from the Philox stream of index s. Same errors. */
cmaes_status cmaes_create_batch(int count, const int* n, const int* lambda,
                                const double* const* x0, const double* sigma0,
                                uint64_t seed, const cmaes_options* opt,
                                cmaes_t* out);

/* Number of searches in the handle. */
int cmaes_count(cmaes_t h);

/* Built-in objective of search s. Q: n*n column-major orthogonal rotation
 * (ignored for SPHERE, may be NULL); lambda_diag: n (ELLIPSOID only); xstar: n.
 * Copied to the device. Errors: EINVAL (bad kind, NULL array it needs). */
cmaes_status cmaes_set_problem(cmaes_t h, int s, int kind, const double* Q,
                               const double* lambda_diag, const double* xstar);

/* Samples the next generation of search s and copies its points to X_host
 * (n*lambda doubles, caller-allocated; lambda from cmaes_query). Must be
 * followed by cmaes_tell before the next ask. Errors: ESTATE (search done or
 * an ask pending). */
cmaes_status cmaes_ask(cmaes_t h, int s, double* X_host);

/* Like cmaes_ask but returns the device address of the n x lambda panel
 * (leading dimension returned in *ld). Valid until the next tell. */
cmaes_status cmaes_ask_device(cmaes_t h, int s, const double** X_dev, int* ld);

/* Completes the pending generation of search s with the objective values
 * f_host (lambda doubles). NaN and +-inf are accepted; NaN ranks as +inf and
 * ties rank by candidate index. Runs the update, the lazy eigendecomposition,
 * the stop tests and a restart if one fires. Errors: ESTATE (no ask pending). */
cmaes_status cmaes_tell(cmaes_t h, int s, const double* f_host);

/* Runs `generations` full generations of every search that is not done, with
 * the built-in objectives, asynchronously on `stream` (a cudaStream_t; NULL
 * selects the handle's own non-blocking stream, which does not order with the
 * legacy default stream). The work is ordered after earlier work of the
 * handle and later calls are ordered after it. Searches that finish stop
 * consuming work. Errors: EINVAL (a search without an objective), ESTATE (an
 * ask is pending). */
cmaes_status cmaes_step_batch(cmaes_t h, int generations, void* stream);

/* Waits for all work of the handle. */
cmaes_status cmaes_sync(cmaes_t h);

/* Asynchronous, batched ask / tell for an external objective over searches
 * [s0, s1), for a costly f evaluated on the host while the device works on
 * other searches (the paper's black-box setting, §1, §4.1). Both calls only
 * enqueue work on `stream` (NULL: the handle's stream) and return; the caller
 * synchronises the stream before reading or reusing the host buffers. Host
 * buffers should be pinned (cudaHostAlloc) for the copies to overlap; pageable
 * memory works but copies synchronously.
 *
 * cmaes_ask_async samples the searches (searches that are done keep their last
 * points) and copies, per search i = s - s0:
 *   X[i]            host, n x lambda_cap doubles, column-major, ld n: the
 *                   panel allocated at creation (lambda_cap = lambda0 *
 *                   2^max_restarts with ipop_double, else lambda0); the
 *                   current points are its first lambda columns;
 *   lam_done[2i]    the current lambda, lam_done[2i + 1] the done flag.
 * cmaes_tell_async copies f[i] (host, lambda_cap doubles, the first lambda
 * used) and enqueues the rest of the generation (rank, update, covariance,
 * eigendecomposition, stop and restart) for the range.
 * Searches of one range must stay on one stream until its tell; other calls
 * on those searches wait for the caller's synchronisation.
 * Errors: EINVAL (range, NULL), ESTATE (ask pending / tell without ask). */
cmaes_status cmaes_ask_async(cmaes_t h, int s0, int s1, double* const* X,
                             int* lam_done, void* stream);
cmaes_status cmaes_tell_async(cmaes_t h, int s0, int s1, const double* const* f,
                              void* stream);

/* Forces Algorithm 2's restart of search s now (lambda doubled if
 * ipop_double); also resumes a search paused by restart_hold (done = 2).
 * Errors: ESTATE (search done for good, ask pending, or a doubled lambda
 * beyond the panels allocated at creation). */
cmaes_status cmaes_restart(cmaes_t h, int s);

/* Best sampled point over all descents of search s (x: n doubles, may be
 * NULL) and its value. Synchronises. */
cmaes_status cmaes_best(cmaes_t h, int s, double* x, double* f);

/* Snapshot / restore of search s (see cmaes_state). Synchronises. On restore
 * lambda must lie in [lambda0, lambda0 * 2^max_restarts] (the capacity the
 * search was created with; lambda0 alone when ipop_double = 0), and a finite
 * sigma must be positive. A non-finite sigma or m is accepted (a checkpoint of
 * a broken state): the next generation's stop test restarts or ends the
 * search and the next status read returns CMAES_ENUMERIC once. */
cmaes_status cmaes_get_state(cmaes_t h, int s, cmaes_state* st);
cmaes_status cmaes_set_state(cmaes_t h, int s, const cmaes_state* st);

/* Points, objective values and rank order of the last completed generation
 * of search s (X: n*lambda, f: lambda, order: lambda; each may be NULL).
 * order[r] is the candidate of rank r. Synchronises. */
cmaes_status cmaes_get_generation(cmaes_t h, int s, double* X, double* f,
                                  int* order);

/* Current lambda, generation, descent number and stop flags of search s (any
 * pointer may be NULL). *done is 1 once the search has ended, 2 while a
 * descent that stopped waits for cmaes_restart (restart_hold), else 0.
 * Synchronises. */
cmaes_status cmaes_query(cmaes_t h, int s, int* lambda, int* gen, int* restart,
                         int* flags, int* done);

/* Per-phase device time. When enabled, cmaes_step_batch records CUDA events
 * around each phase on the stream it launches on; cmaes_phase_times
 * synchronises and returns the accumulated milliseconds and launch counts:
 *   0 sample (z, B D z, x)   1 objective   2 rank + recombination + paths
 *   3 covariance update      4 eigendecomposition   5 stop + restart
 * ms and launches hold 6 entries each (either may be NULL); reset clears. */
cmaes_status cmaes_set_profiling(cmaes_t h, int enable);
cmaes_status cmaes_phase_times(cmaes_t h, double* ms, long long* launches,
                               int reset);

/* Work done by the eigensolver of search s since creation: decompositions,
 * FP64 Jacobi sweeps, plane rotations applied by them, and the FP32 Jacobi
 * sweeps that precede them on the refined route (32 < n <= 4096, every handle
 * precision; zero for other n). Any pointer may be NULL. Synchronises. */
cmaes_status cmaes_eig_stats(cmaes_t h, int s, long long* decompositions,
                             long long* sweeps, long long* rotations,
                             long long* sweeps32);

/* Device time of the stages of the tridiagonal eigensolver route, summed over
 * the generations run with profiling enabled (cmaes_set_profiling): ms[0]
 * Householder reduction, ms[1] eigenvalues (splitting, bisection, ranks),
 * ms[2] eigenvectors of T by inverse iteration, ms[3] Gram-Schmidt inside
 * clusters of close eigenvalues, ms[4] Newton-Schulz orthogonalisation,
 * ms[5] back-transformation and canonical form. ms: host array of 6;
 * reset != 0 zeroes the sums. Zero when
 * no search takes that route. Synchronises with the handle's stream. */
cmaes_status cmaes_eig_stage_times(cmaes_t h, double* ms, int reset);

/* Number of kernel launches issued by the handle since creation. */
long long cmaes_kernel_launches(cmaes_t h);

/* Evaluates a built-in objective on lambda points without allocating any
 * device memory. The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc at that point -- code whose device memory is managed
 * by another component (a framework's caching allocator, a plug-in inside a
 * host application) or loops where the latency and implicit synchronisation
 * of an allocation are not acceptable. It computes the same f as the engine's
 * objective phase, bit for bit.
 *
 *   kind         CMAES_OBJ_ELLIPSOID, _RASTRIGIN or _SPHERE
 *   X            device, n x lambda column-major, leading dimension ld >= n
 *   Q            device, n x n column-major, leading dimension ldq >= n
 *                (not read for SPHERE; may be NULL then)
 *   lambda_diag  device, n (ELLIPSOID only; may be NULL otherwise)
 *   xstar        device, n
 *   f            device, lambda doubles, written
 *   stream       cudaStream_t the kernels are launched on (NULL: legacy default)
 *
 * The intermediate U = Q (X - x*) lives in one static device array of 2^20
 * doubles (8 MiB) that every GPU loading the library keeps until the process
 * exits; ld * lambda above 2^20 is rejected with CMAES_EINVAL (SPHERE needs no
 * scratch and has no limit). All calls share that array: two calls whose
 * kernels overlap on the GPU (different streams, or different threads on the
 * same device) race and give wrong results. Nothing in it needs to start at
 * zero. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture. A reset of
 * the device or of its primary context (cudaDeviceReset) reloads the module
 * and leaves the kept address stale: do not call this entry point after such
 * a reset. The call is asynchronous on `stream`; errors:
 * EINVAL (arguments, size), ECUDA; the text is in cmaes_last_error(NULL). */
cmaes_status cmaes_evaluate_noalloc(int kind, int n, int lambda, const double* X,
                                    int ld, const double* Q, int ldq,
                                    const double* lambda_diag,
                                    const double* xstar, double* f,
                                    void* stream);

/* Fault injection from the host (no counterpart in the paper; for tests of
 * the error paths above, which must not be provoked by faulting the GPU):
 * waits for the handle's stream, then ORs `bits` into the handle's device
 * status word exactly as the device does. bits: 1 = a bounded device wait
 * timed out (later calls return CMAES_ETIMEOUT, sticky), 2 = a search's state
 * became non-finite (the next status read returns CMAES_ENUMERIC once). Other
 * bits: EINVAL. */
cmaes_status cmaes_inject_status(cmaes_t h, int bits);

const char* cmaes_strerror(cmaes_status st);
/* Text of the last error on h (or of the last failed create if h is NULL). */
const char* cmaes_last_error(cmaes_t h);

/* Releases all device and host memory of the handle. NULL is a no-op. */
void cmaes_destroy(cmaes_t h);

#ifdef __cplusplus
}
#endif
#endif /* CMAES_GB300_CMAES_H */
