/*
 * qbx_peaks.h - arithmetic-peak probes of libqbx (measurement aids, not steps of the paper's method).
 *
 * The evaluation kernels of the GIGAQBX path (Wala & Kloeckner, arXiv 1805.06106, Algorithm 4) are
 * bound by FP64 arithmetic (the near-field P2QBXL sums, translations) or, in the mixed-precision modes,
 * partly by FP32 arithmetic.  These probes measure the device's fused multiply-add throughput so that
 * each kernel's achieved rate can be stated as a fraction of a measured peak.
 */
#ifndef QBX_PEAKS_H
#define QBX_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

#define QBX_PEAK_FP64 0
#define QBX_PEAK_FP32 1

/*
 * Measures the FP64 (kind QBX_PEAK_FP64) or FP32 (QBX_PEAK_FP32) fused multiply-add throughput:
 * every thread of a grid of 2, 4 and 8 blocks of 256 threads per SM runs eight independent FMA
 * chains; the best of `reps` timed launches per grid (CUDA events on `stream`, after one warm-up
 * launch) is written to *flops_host in flop/s (an FMA counts as 2).  Allocates 8 bytes of device
 * memory for the duration of the call and synchronizes `stream`.  Up to about 0.1 s per launch.
 * Errors: QBX_ERR_INVALID_ARG (bad kind, reps < 1, NULL output), QBX_ERR_OOM, QBX_ERR_CUDA.
 */
int qbx_peak_flops(int kind, int reps, double *flops_host, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QBX_PEAKS_H */
