/*
 * nrmg_peak.h -- FMA throughput microbenchmark shipped with libnrmg.so.
 *
 * The paper has no counterpart: this call measures the denominator of the roofline
 * fraction that the solver's kernels are reported against (the solver path is bound by
 * FP64 arithmetic, and the GPU's FP64/FP32 FMA rates are not published for this part).
 *
 * nrmg_peak_fma runs a kernel of independent FMA chains (8 per thread, `iters` rounds) on
 * every SM of the current device, on `cuda_stream` (cudaStream_t as void*, NULL = legacy
 * default stream), times it with CUDA events and writes the achieved rate in FLOP/s
 * (2 flops per FMA) to *flops_per_s.  precision: 0 = FP64 (DFMA), 1 = FP32 (FFMA).
 * Synchronizes the stream.  Returns 0 on success, 1 on an invalid argument, 2 on a CUDA
 * error.  Allocates a small device buffer (one value per thread) for the kernel's results.
 */
#ifndef NRMG_PEAK_H
#define NRMG_PEAK_H

#ifdef __cplusplus
extern "C" {
#endif

int nrmg_peak_fma(int precision, int iters, void *cuda_stream, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif
