// noalloc.cu -- objective evaluation that allocates no device memory.
//
// Some callers cannot allocate: code that runs while another component owns
// the device's memory budget (a framework's caching allocator, a plug-in
// inside a host application), or latency-bound loops in which a cudaMalloc and
// the synchronisation it implies are not acceptable. For them this file
// evaluates the built-in objectives on caller-provided device buffers, with the
// one intermediate it needs (U = Q (X - x*)) held in a file-scope device array
// of fixed size instead of engine-allocated scratch. The arithmetic is the same
// as the engine's objective phase (k_gemm_objective + k_colreduce_f): the same
// 64 x 64 FP64 GEMM tile and the same per-column reduction order, so results
// agree bit for bit.
#include <cmath>
#include <cstdio>
#include <string>

#include "../../include/cmaes.h"
#include "device_common.cuh"

namespace cmaes_gb300 {
namespace {

// Scratch for U: 2^20 doubles (8 MiB). Every GPU that loads this library keeps
// it until the process exits.
constexpr long long kEvalScratchDoubles = 1LL << 20;
__device__ __align__(256) double g_eval_scratch[kEvalScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(256) k_noalloc_rotate(int n, int lam, int ld, const double* X,
                                                        const double* Q, int ldq,
                                                        const double* xstar, double* U) {
  __shared__ GemmSmem sm;
  const int mt = ceil_div(n, kGBM);
  const int i0 = (blockIdx.x % mt) * kGBM, j0 = (blockIdx.x / mt) * kGBN;
  gemm_tile_f64<true, true>(
      n, lam, n, i0, j0,
      [=] __device__(int i, int k) { return Q[i + static_cast<long long>(ldq) * k]; },
      [=] __device__(int k, int j) { return X[k + static_cast<long long>(ld) * j] - xstar[k]; },
      [=] __device__(int i, int j, double acc) { U[i + static_cast<long long>(ld) * j] = acc; },
      sm);
}

__global__ void __launch_bounds__(256) k_noalloc_reduce(int kind, int n, int lam, int ld,
                                                        const double* X, const double* U,
                                                        const double* lamdiag,
                                                        const double* xstar, double* f) {
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= lam) return;
  double acc = 0.0;
  if (kind == CMAES_OBJ_SPHERE) {
    const double* x = X + static_cast<long long>(ld) * k;
    for (int i = lane; i < n; i += 32) {
      const double r = x[i] - xstar[i];
      acc += r * r;
    }
  } else if (kind == CMAES_OBJ_ELLIPSOID) {
    const double* u = U + static_cast<long long>(ld) * k;
    for (int i = lane; i < n; i += 32) acc += lamdiag[i] * u[i] * u[i];
  } else {
    const double* u = U + static_cast<long long>(ld) * k;
    for (int i = lane; i < n; i += 32) acc += u[i] * u[i] - 10.0 * cos((2.0 * 3.141592653589793) * u[i]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) f[k] = (kind == CMAES_OBJ_RASTRIGIN) ? 10.0 * n + acc : acc;
}

cmaes_status noalloc_fail(cmaes_status st, const std::string& msg) {
  set_global_error(msg.c_str());  // readable through cmaes_last_error(NULL)
  return st;
}

}  // namespace
}  // namespace cmaes_gb300

using namespace cmaes_gb300;

extern "C" cmaes_status cmaes_evaluate_noalloc(int kind, int n, int lambda, const double* X, int ld,
                                               const double* Q, int ldq, const double* lambda_diag,
                                               const double* xstar, double* f, void* stream) {
  if (kind < CMAES_OBJ_ELLIPSOID || kind > CMAES_OBJ_SPHERE)
    return noalloc_fail(CMAES_EINVAL, "cmaes_evaluate_noalloc: unknown objective kind");
  if (n < 1 || lambda < 1 || ld < n || !X || !xstar || !f)
    return noalloc_fail(CMAES_EINVAL, "cmaes_evaluate_noalloc: bad size or NULL buffer");
  if (kind != CMAES_OBJ_SPHERE && (!Q || ldq < n))
    return noalloc_fail(CMAES_EINVAL, "cmaes_evaluate_noalloc: Q missing or ldq < n");
  if (kind == CMAES_OBJ_ELLIPSOID && !lambda_diag)
    return noalloc_fail(CMAES_EINVAL, "cmaes_evaluate_noalloc: lambda_diag missing");
  const bool rotated = kind != CMAES_OBJ_SPHERE;
  if (rotated && static_cast<long long>(ld) * lambda > kEvalScratchDoubles) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "cmaes_evaluate_noalloc: ld * lambda = %lld exceeds the %lld-double scratch "
             "(use the engine's allocating path for larger panels)",
             static_cast<long long>(ld) * lambda, kEvalScratchDoubles);
    return noalloc_fail(CMAES_EINVAL, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(CMAES_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CMAES_EUNSUPPORTED, "device index too large");
  // One-time set-up per device, with that device current: the host-side name
  // of the array is not a device address, so ask the runtime for it.
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess) return noalloc_fail(CMAES_ECUDA, cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  double* U = g_scratch_addr[dev];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (rotated) {
    const int tiles = ceil_div(n, kGBM) * ceil_div(lambda, kGBN);
    k_noalloc_rotate<<<tiles, 256, 0, st>>>(n, lambda, ld, X, Q, ldq, xstar, U);
  }
  k_noalloc_reduce<<<ceil_div(lambda, 8), 256, 0, st>>>(kind, n, lambda, ld, X, U, lambda_diag, xstar, f);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(CMAES_ECUDA, cudaGetErrorString(e));
  return CMAES_OK;
}
