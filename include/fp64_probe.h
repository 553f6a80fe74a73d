/* fp64_probe.h -- FP64 pipe throughput probe of the GPU (a measurement tool of this library,
 * not a step of the paper's method; the paper has no counterpart).
 *
 * The local solves of the overlapped RBF-FD method are FP64 work (§4.3: one factorization of
 * cost O((n+M)^3) per stencil).  This probe measures what the GPU's FP64 units deliver, so
 * that the roofline of those kernels has a measured denominator beside the nominal one, and
 * whether the FP64 tensor-core instruction (DMMA, mma.sync m8n8k4 f64) beats plain FMAs.
 *
 * fp64_probe_run -- time one launch of the probe kernel on `stream` with CUDA events.
 *   kind     0: independent DFMA chains (8 per thread), 1: DMMA m8n8k4 tiles (4 independent
 *            accumulators per warp), 2: both kernels at once, DFMA on half the SMs' worth of
 *            blocks and DMMA on the other half (does mixing add throughput?)
 *   iters    inner iterations per thread (>= 1; the work is iters x the per-iteration flops)
 *   tflops   out: FP64 TFLOP/s of the launch (FMA = 2 flops; a DMMA = 8 x 8 x 4 FMAs)
 *   ms       out: the launch's duration
 * The kernels use no memory beyond one store per thread to a 1 MB device buffer the library
 * allocates once per device (so the compiler keeps the arithmetic); they wait on nothing.
 * Returns 0, or -1 for bad arguments, -6 for a CUDA error. */
#ifndef FP64_PROBE_H
#define FP64_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif
int fp64_probe_run(int kind, int iters, void* stream, double* tflops, float* ms);
#ifdef __cplusplus
}
#endif
#endif
