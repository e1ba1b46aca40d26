/*
 * cmaes_ozaki.h -- the engine's FP64-accurate matrix product on the BF16
 * tensor cores, exported for testing and measurement.
 *
 * The paper rewrites the linear algebra of a CMA-ES generation as Level-3
 * BLAS calls in FP64 (§3.1: dgemm for the sampling and the covariance update,
 * dsyev for the eigendecomposition). On GB300 FP64 runs on the CUDA cores at
 * about 1.25 TFLOP/s, so the eigensolver's long products are computed as
 * exact sums of BF16 digit-plane products on the tensor cores instead (the
 * error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012): each row of A
 * and each column of B is rounded once to a 54-bit fixed-point number relative
 * to its own largest entry, and the product of those numbers is formed with
 * no further rounding before the final FP64 value. This entry point runs that
 * product on its own.
 */
#ifndef CMAES_GB300_OZAKI_H
#define CMAES_GB300_OZAKI_H
#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * A * B + beta * C on the current device, FP64 in and out.
 *
 * A: device pointer, M x K, column-major with leading dimension lda >= M.
 * B: device pointer, K x N, column-major, ldb >= K.
 * C: device pointer, M x N, column-major, ldc >= M; read only if beta != 0.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * The caller owns all three arrays. The call allocates and frees its own
 * workspace (about 14 bytes per element of A and B) and returns after the
 * product is complete.
 *
 * Accuracy: with 2^a the power of two bounding row i of A (2^a < 2 x its
 * largest magnitude) and 2^b the one bounding column j of B, every entry is
 * represented to within 2^(a-55) (resp. 2^(b-55)); the digit products
 * dropped by the scheme add less than 6 * 2^(a+b-54) per term of the K sum;
 * everything else is summed exactly down to 2^-40 of the leading digit
 * product, and the result is rounded once to FP64. Entries below 2^-1022
 * count as zero.
 *
 * Returns 0 on success, 1 on a bad argument, 2 if the workspace cannot be
 * allocated, 3 on a CUDA error, 4 if a device wait ran out (about 1 s). */
int cmaes_ozaki_dgemm(int M, int N, int K, double alpha, const double* A, long long lda,
                      const double* B, long long ldb, double beta, double* C, long long ldc,
                      void* stream);

#ifdef __cplusplus
}
#endif
#endif
