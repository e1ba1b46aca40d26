/*
 * cmaes_probe.h -- arithmetic-rate probe used to state the FP64 and FP32
 * roofs of the engine's ALU-bound kernels (the eigensolver and the FP64
 * GEMMs). Not part of the method: the paper has no counterpart; it measures
 * the device the benchmark runs on.
 */
#ifndef CMAES_GB300_PROBE_H
#define CMAES_GB300_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Runs dependent-chain FMA kernels (8 independent chains per thread, 256
 * threads per block, blocks_per_sm blocks on every SM) on the current device
 * and returns the best of `repeats` timed launches in TFLOP/s (2 flops per
 * FMA). precision: 64 (FP64 DFMA) or 32 (FP32 FFMA). Returns 0 on success,
 * 1 on a bad argument, 3 on a CUDA error. */
int cmaes_probe_fma_tflops(int precision, int blocks_per_sm, int repeats, double* tflops);

#ifdef __cplusplus
}
#endif
#endif
