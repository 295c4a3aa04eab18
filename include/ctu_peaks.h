/* ctu_peaks.h -- measurement aid beside the CTU library, built as a library
 * of its own (libctu_peaks.so) and not part of libctu.so.  The paper has no
 * counterpart: it measures the non-tensor pipes whose peaks the step's
 * arithmetic roofline is read against. */
#ifndef CTU_PEAKS_H
#define CTU_PEAKS_H

#include "ctu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FMA-throughput microbenchmark of the non-tensor pipes on the current
 * device: every thread of a grid of 16 blocks of 256 threads per SM runs 8
 * independent chains of `iters` fused multiply-adds in float32 (fp64 = 0) or
 * float64 (fp64 = 1); *flops_per_s = 2 x FMAs / CUDA-event time of the timed
 * launch (after one shorter warm-up launch).  Synchronises the stream;
 * allocates and frees a small scratch array.  Returns CTU_EINVAL for a null
 * output or iters < 1, CTU_ECUDA on a CUDA error. */
ctu_status ctu_fma_peak(int fp64, int iters, double *flops_per_s, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CTU_PEAKS_H */
