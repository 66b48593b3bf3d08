/*
 * Measurement helper of the tpcfit library (the paper has no counterpart):
 * measures the arithmetic pipes that bound the track fit on this GPU, so that
 * throughput can be stated as a fraction of a measured peak.
 */
#ifndef TPCFIT_PROBE_H
#define TPCFIT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Run dependent-chain FMA loops (8 independent chains per thread, 8 blocks of
 * 256 threads per SM) on `device` and report the sustained throughput of
 * FP64 fused multiply-adds and FP32 fused multiply-adds, in lane-operations
 * per second (one FMA of one thread = 1), plus the SM clock the device
 * reports (kHz).  Any output pointer may be NULL.  Takes ~50 ms.  Returns 0,
 * or a negative TPCFIT_E_* code (TPCFIT_E_NODEV without a device). */
int tpcfit_probe_fma_rates(int device, double *fp64_fma_per_s, double *fp32_fma_per_s, int *sm_clock_khz);

#ifdef __cplusplus
}
#endif
#endif /* TPCFIT_PROBE_H */
