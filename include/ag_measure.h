/* ag_measure.h — measurement utility of libaerialgb (not part of the
 * simulation).
 *
 * The fused fleet step (ag_step) is bound by plain FP32 arithmetic on the CUDA
 * cores: there is no dense contraction for the tensor cores. Its roofline
 * denominator is derived from the unit counts, SMs x 128 FP32 lanes x 2 FLOP
 * per FMA x the maximum SM clock. ag_measure_fp32_peak measures what a kernel
 * made of nothing but independent FMAs reaches on the current device, once in
 * scalar fmaf form and once in the packed FP32x2 form (__ffma2_rn) that the
 * fused step uses, as a check of that derivation. The errors follow ag.h.
 */
#ifndef AG_MEASURE_H
#define AG_MEASURE_H

#include "ag.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double scalar_tflops; /* FP32 FLOP/s / 1e12, scalar FMA chains (2 FLOP per FMA) */
  double packed_tflops; /* the same with packed FP32x2 FMAs (4 FLOP per instruction) */
  double scalar_ms;     /* best launch time of the scalar kernel [ms] */
  double packed_ms;     /* best launch time of the packed kernel [ms] */
  uint32_t grid;        /* blocks per launch: SMs x resident blocks per SM */
  uint32_t block;       /* threads per block */
} ag_fp32_peak;

/* Runs both FMA-chain kernels on the current CUDA device, on the stream
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream), and writes
 * the best of `reps` timed launches of each (after one warm-up launch) to
 * *out. `iters` (1 .. 1,000,000) sets the work: every thread performs
 * 128 x iters FMAs (scalar) or packed FMAs. Synchronous: the call returns
 * after the last launch has finished. It allocates and frees one device
 * buffer of grid x block floats. AG_ERR_INVALID (nothing launched) when out
 * is NULL or iters or reps (1 .. 100) is out of range; AG_ERR_CUDA when a
 * CUDA call fails (ag_last_error(NULL) gives the message). */
ag_status ag_measure_fp32_peak(void* cuda_stream, uint32_t iters, uint32_t reps, ag_fp32_peak* out);

#ifdef __cplusplus
}
#endif

#endif /* AG_MEASURE_H */
