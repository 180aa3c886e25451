/*
 * Measured arithmetic peaks of a GPU: the denominators of the pbfmm
 * kernels' rooflines (the near field and check potentials are bound by the
 * FP32 fused multiply-add pipe and the MUFU reciprocal-square-root and
 * exponential units; the box operators by the tensor cores' TF32 rate; the
 * all-FP64 path by FP64 arithmetic).  Not part of the solver's interface.
 */
#ifndef PBFMM_PEAKS_H
#define PBFMM_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Runs one short microbenchmark per pipe on CUDA device `device` (about
 * 0.2 s in all; CUDA events on a private stream, one warm-up launch each)
 * and writes out[7]:
 *   out[0]  FP32 fused multiply-add, TFLOP/s (2 FLOP per FMA)
 *   out[1]  MUFU rsqrt.approx.ftz.f32, 10^12 results/s
 *   out[2]  MUFU ex2.approx.ftz.f32, 10^12 results/s
 *   out[3]  FP64 fused multiply-add, TFLOP/s
 *   out[4]  tcgen05.mma kind::tf32 (M 128, N 256, operands in shared
 *           memory, FP32 accumulator in TMEM), dense TFLOP/s
 *   out[5]  the same loop with kind::f16, BF16 operands, TFLOP/s
 *   out[6]  packed FP32 fused multiply-add (fma.rn.f32x2, two FMAs per
 *           instruction), TFLOP/s
 * The rates hold at whatever SM clock the GPU ran (sample it alongside).
 * Returns PB_OK, PB_ECUDA, or PB_ETIMEOUT if a tensor-core wait gave up. */
int pbfmm_measure_peaks(int device, double* out);

#ifdef __cplusplus
}
#endif

#endif /* PBFMM_PEAKS_H */
