/*
 * gaps_peaks.h - throughput of the GPU's arithmetic pipes, measured by the
 * library's own microbenchmarks. A measurement helper for the shower's
 * roofline (the paper has no counterpart: it reports no roofline); it is not
 * on the shower's path.
 */
#ifndef GAPS_PEAKS_H
#define GAPS_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

#define GAPS_PEAK_FFMA 0  /* FP32 fused multiply-add instructions per lane */
#define GAPS_PEAK_DFMA 1  /* FP64 fused multiply-add instructions per lane */
#define GAPS_PEAK_MUFU 2  /* special-function (ex2, lg2) instructions per lane */
#define GAPS_PEAK_IMAD 3  /* 32-bit products with both halves kept (a Philox round's
                             multiply), with an add and a xor, per lane */

/* Runs dependent-chain microbenchmarks of one instruction kind on the current
 * device (8 independent chains per thread, 2048 threads per SM; per thread
 * `iters` x 128 instructions, or `iters` x 64 products for GAPS_PEAK_IMAD;
 * one warm-up launch and the best of three timed launches on `stream`,
 * synchronised). Writes the instruction throughput
 * summed over all lanes (per second) to *ops_per_s and the best launch's
 * duration in ms to *ms (may be NULL). Allocates and frees one scratch
 * buffer. Returns 0, -1 for a bad kind or iters (1 .. 2^20), -5 on a CUDA
 * error, -6 without a device. The clock is whatever the GPU runs at: the
 * caller samples it. */
int gaps_alu_peak(int kind, int iters, double* ops_per_s, double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GAPS_PEAKS_H */
