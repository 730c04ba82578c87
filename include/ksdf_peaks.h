/*
 * ksdf_peaks.h -- C ABI of libksdf_peaks.so, the throughput probes that give the roofline denominators of
 * the Kernel-SDF kernels on the GPU they run on (the paper has no counterpart: this is measurement
 * instrumentation, kept out of libksdf.so).
 *
 * ksdf_peaks_measure(unit, stream, rate) runs one probe on the current CUDA device: a warm-up launch, then
 * one launch timed with CUDA events on `stream` (a cudaStream_t; NULL = legacy default), and writes the
 * achieved rate to *rate (host).  The call synchronises the stream and allocates (and frees) 64 bytes of
 * device memory.  Units and what *rate means:
 *   KSDF_PEAK_FP64_DFMA     FP64 FLOP/s / 1e12 (2 per DFMA): four dependent DFMA chains per thread,
 *                           512 threads per SM
 *   KSDF_PEAK_FP32_FFMA     FP32 FFMA instructions per second per lane / 1e12 (lane operations, one per FMA;
 *                           the unit the kernels' FP32 operation counts use): eight chains per thread,
 *                           2 x 1024 threads per SM
 *   KSDF_PEAK_FP32X2_FFMA   FP32 lane FMAs per second / 1e12 issued as packed fma.rn.f32x2 (two per
 *                           instruction): eight chains per thread, 2 x 1024 threads per SM
 *   KSDF_PEAK_MUFU_EX2      ex2.approx operations per second / 1e12: eight chains per thread, 2 x 1024
 *                           threads per SM
 *   KSDF_PEAK_TF32_TCGEN05  dense TF32 tensor FLOP/s / 1e12 of tcgen05.mma kind::tf32 (M = 128, N = 256,
 *                           K = 8, FP32 accumulation in TMEM), one CTA per SM issuing 8,192 MMAs
 * Returns 0 on success; 1 for a NULL rate or an unknown unit, 2 if a CUDA call failed, 7 if the MMA
 * completion wait of the tensor-core probe gave up (bounded spin; the kernel returns after releasing its
 * TMEM).  ksdf_peaks_last_error() gives a message.
 */
#ifndef KSDF_PEAKS_H
#define KSDF_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  KSDF_PEAK_FP64_DFMA = 0,
  KSDF_PEAK_FP32_FFMA = 1,
  KSDF_PEAK_MUFU_EX2 = 2,
  KSDF_PEAK_TF32_TCGEN05 = 3,
  KSDF_PEAK_FP32X2_FFMA = 4
};

int ksdf_peaks_measure(int unit, void* stream, double* rate);
const char* ksdf_peaks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
