/*
 * md_bench.h -- measurement helpers of the GB300 MD library (not part of the
 * method of Colberg & Hoefling; they give its roofline a measured denominator).
 */
#ifndef MD_GB300_BENCH_H
#define MD_GB300_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic peak of the current GPU's CUDA cores, measured: every thread of
 * four full waves of 256-thread blocks on every SM runs 8 independent chains
 * of 16 * iters fused multiply-adds in precision 0 (FP64) or 2 (FP32); the
 * fastest of 3 timed launches (CUDA events, legacy default stream, after one
 * warm-up launch) gives *tflops = 2 * FMAs / time, in TFLOP/s, and *ms its
 * duration (may be NULL).  Synchronises the device.  Returns 0, 1 (bad
 * argument: null tflops, iters < 1, another precision) or 3 (a CUDA call
 * failed).  Changes no clock or other setting of the GPU. */
int md_fma_peak(int32_t precision, int64_t iters, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* MD_GB300_BENCH_H */
