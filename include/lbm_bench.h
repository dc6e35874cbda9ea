/*
 * lbm_bench.h -- measurement helpers of libmrtlbm.so that are not part of the
 * method: arithmetic-throughput probes that give the ALU rooflines of the
 * step kernels a measured denominator (the paper has no counterpart).
 *
 * Same conventions as lbm.h: 0 on success, a negative LBM_* code otherwise.
 */
#ifndef LBM_BENCH_H
#define LBM_BENCH_H

#ifdef __cplusplus
extern "C" {
#endif

/* Throughput of dependent-free fused multiply-adds on device `device`
 * (-1: the current one), timed with CUDA events over `reps` launches after
 * one warm-up launch; each launch covers every SM with independent FMA
 * chains.  kind 0: FP64 (fma.rn.f64), 1: FP32 (fma.rn.f32), 2: packed
 * FP32x2 (fma.rn.f32x2, two FMAs per instruction).  *fma_per_s receives
 * thread-level FMA operations per second (a packed instruction counts two;
 * FLOP/s = 2 x this) and *inst_per_s (may be NULL) thread-level
 * instructions per second.  Allocates and frees a small device buffer; runs
 * on the legacy default stream and synchronises the device.
 * Errors: LBM_ERR_ARG (kind, reps < 1 or NULL output), LBM_ERR_CUDA. */
int lbm_bench_fma_peak(int kind, int device, int reps, double *fma_per_s, double *inst_per_s);

#ifdef __cplusplus
}
#endif
#endif
