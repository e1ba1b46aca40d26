// kernels_ozaki.cu -- the general FP64-accurate product C = alpha A B + beta C
// on the BF16 tensor cores (digit planes and bucket sums of ozaki.cuh), used
// by include/cmaes_ozaki.h and by the eigensolver's Gram products.
#include <cuda_runtime.h>
#include "../../include/cmaes_ozaki.h"
#include "engine.h"
#include "ozaki.cuh"

namespace cmaes_gb300 {

// One operand to pack: x(r, k) = src[r * sr + k * sk], r < R, k < K.
struct OzPackJob {
  const double* src;
  long long sr, sk;
  int R, K, nks;
  unsigned char* out;
  int* e;
  int block0;  // first CTA of this job in the launch
};

__global__ void __launch_bounds__(kOzNT) k_oz_pack(const OzPackJob* jobs, int njobs) {
  __shared__ int sh_e[64];
  int j = 0;
  while (j + 1 < njobs && jobs[j + 1].block0 <= static_cast<int>(blockIdx.x)) ++j;
  const OzPackJob J = jobs[j];
  const int rb = static_cast<int>(blockIdx.x) - J.block0;
  oz_pack_block(J.src, J.sr, J.sk, J.R, J.K, rb, J.nks, J.out, J.e, sh_e);
}

// C (M x N, column-major, ldc) = alpha * A B + beta * C from packed A (M rows)
// and B (N rows), K = nks * 32. One 128 x 64 output tile per CTA.
struct OzGemmJob {
  const unsigned char* a;
  const int* ea;
  const unsigned char* b;
  const int* eb;
  int M, N, nks;
  double* c;
  long long ldc;
  double alpha, beta;
};

__global__ void __launch_bounds__(kOzNT, 1) k_oz_gemm(const OzGemmJob* job, int* err) {
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[5];
  __shared__ uint32_t tslot;
  const OzGemmJob J = *job;
  const int tn_count = (J.N + kOzBN - 1) / kOzBN;
  const int tm = static_cast<int>(blockIdx.x) / tn_count, tn = static_cast<int>(blockIdx.x) % tn_count;
  OzCtx cx;
  oz_begin(cx, dyn, bar, &tslot);
  long long W[32];
  float L[32];
  const bool ok = oz_tile(cx, J.a, oz_pitch(J.nks), 2 * tm, J.b, oz_pitch(J.nks), tn, J.nks, W, L);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, kDevErrTimeout);
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = tm * kOzBM + 32 * (warp & 3) + lane;
    const int jb = tn * kOzBN + 32 * (warp >> 2);
    if (i < J.M) {
      const int ea = J.ea[i];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = jb + q;
        if (j >= J.N) continue;
        const double v = oz_value(W[q], L[q], ea, J.eb[j]);
        double* cp = J.c + i + J.ldc * j;
        *cp = J.beta == 0.0 ? J.alpha * v : fma(J.alpha, v, J.beta * *cp);
      }
    }
  }
  oz_end(cx);
}

}  // namespace cmaes_gb300

using namespace cmaes_gb300;

extern "C" int cmaes_ozaki_dgemm(int M, int N, int K, double alpha, const double* A, long long lda,
                                 const double* B, long long ldb, double beta, double* C, long long ldc,
                                 void* stream) {
  if (M < 0 || N < 0 || K < 0) return 1;
  if (M == 0 || N == 0) return 0;
  if (!A || !B || !C || lda < M || ldb < K || ldc < M) return 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nks = oz_nks(K);
  const size_t abytes = oz_bytes(M, K), bbytes = oz_bytes(N, K);
  const int mpad = oz_rows_padded(M), npad = oz_rows_padded(N);
  unsigned char* ws = nullptr;
  const size_t jobs_off = abytes + bbytes + sizeof(int) * (mpad + npad);
  const size_t jobs_at = (jobs_off + 255) / 256 * 256;
  const size_t total = jobs_at + sizeof(OzPackJob) * 2 + sizeof(OzGemmJob) + sizeof(int);
  if (cudaMalloc(&ws, total) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  unsigned char* pa = ws;
  unsigned char* pb = ws + abytes;
  int* ea = reinterpret_cast<int*>(ws + abytes + bbytes);
  int* eb = ea + mpad;
  OzPackJob pj[2];
  // A: row i, K index k at A[i + lda k]; B: row j (a column of B), k at B[k + ldb j]
  pj[0] = OzPackJob{A, 1, lda, M, K, nks, pa, ea, 0};
  pj[1] = OzPackJob{B, ldb, 1, N, K, nks, pb, eb, mpad / 64};
  OzGemmJob gj{pa, ea, pb, eb, M, N, nks, C, ldc, alpha, beta};
  OzPackJob* d_pj = reinterpret_cast<OzPackJob*>(ws + jobs_at);
  OzGemmJob* d_gj = reinterpret_cast<OzGemmJob*>(d_pj + 2);
  int* d_err = reinterpret_cast<int*>(d_gj + 1);
  int rc = 0;
  int herr = 0;
  if (cudaMemcpyAsync(d_pj, pj, sizeof(pj), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_gj, &gj, sizeof(gj), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) {
    rc = 3;
  } else {
    k_oz_pack<<<mpad / 64 + npad / 64, kOzNT, 0, st>>>(d_pj, 2);
    cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
    const int tiles = (mpad / kOzBM) * ((N + kOzBN - 1) / kOzBN);
    k_oz_gemm<<<tiles, kOzNT, kOzSmem, st>>>(d_gj, d_err);
    if (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = 3;
    else if (herr)
      rc = 4;
  }
  if (cudaGetLastError() != cudaSuccess) rc = 3;
  cudaFree(ws);
  return rc;
}
