/*
 * md_probe.h -- measurement probe shipped with the MD library.
 *
 * The roofline of the plain FP64 path (the precision the paper computes in,
 * Sec. 2 and Table 1) needs the GPU's FP64 arithmetic rate, which on this part
 * is a small fraction of its FP32 rate.  This probe measures it instead of
 * assuming a nominal figure: a kernel of independent FP64 fused multiply-add
 * chains, sized to every SM, timed with CUDA events.  It is not part of the
 * MD computation.
 */
#ifndef MD_PROBE_H
#define MD_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 FMA rate.  Launches `blocks_per_sm` x (SM count) blocks of 256 threads,
 * each thread running 8 independent chains of `iters` FP64 FMAs (a = a * b + c,
 * with operands that keep the values finite), and times the launch with CUDA
 * events on `stream`.  Writes the rate in TFLOP/s (2 flops per FMA) to
 * *tflops and the launch time in milliseconds to *ms (host pointers).
 * Synchronises `stream`.  Returns 0 on success, -1 for bad arguments
 * (iters < 1, blocks_per_sm outside 1..32, NULL outputs), -2 on a CUDA error. */
int md_probe_fp64_fma(int64_t iters, int32_t blocks_per_sm, double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MD_PROBE_H */
