/* ag_measure.h — measurement utilities of libaerialgb (not part of the
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

typedef struct {
  uint32_t sm_count;          /* streaming multiprocessors (cudaDevAttrMultiProcessorCount) */
  uint32_t fp32_lanes_per_sm; /* FP32 FMA lanes per SM of the compute capability (128 on sm_10x) */
  uint32_t max_sm_clock_khz;  /* peak SM clock (cudaDevAttrClockRate) */
  uint32_t cc_major, cc_minor;
  double tflops;              /* sm_count x lanes x 2 FLOP per FMA x clock / 1e12 */
} ag_alu_peak;

/* The derived FP32 CUDA-core peak of CUDA device `device`, from the device's
 * own attributes: SM count and peak SM clock as the driver reports them,
 * FP32 lanes per SM from the compute capability (64 on 6.0, 7.x and 8.0;
 * 128 on every other capability from 6.1 on). AG_ERR_INVALID for a NULL out
 * or a capability below 6.0; AG_ERR_CUDA when a query fails. No launch, no
 * allocation. */
ag_status ag_query_alu_peak(int device, ag_alu_peak* out);

/* The ray caster of ag_render_depth (include/ag.h; Sec. III depth cameras,
 * Sec. VII kernel-based ray casting), same arguments and results, with the
 * slab intervals' three reciprocals per pixel and box correctly rounded
 * (IEEE division) instead of the fast approximate reciprocal that
 * ag_render_depth uses. It exists to measure how many pixels the
 * approximation moves: it is not faster and not otherwise different. */
ag_status ag_render_depth_ieee(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                               const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams, float* depth);

/* The number of (environment, step) collision tests the last ag_step of the
 * context ran, into *tests (host). The method tests every environment
 * against every box after every step (n_envs x steps); the fused step skips
 * a test while the vehicle has moved less from its last exact test than
 * that test's clearance to the nearest box (minus a rounding slack), which
 * changes no decision. This count is the work a launch performed, against
 * which its performed-work ALU fraction is stated. 0 before the first
 * ag_step; the unfused path does not count. Synchronises the context's
 * stream. AG_ERR_INVALID for a NULL tests. */
ag_status ag_collision_tests_run(ag_ctx* ctx, uint64_t* tests);

/* Counts the (pixel, box) pairs that ag_render_depth, with the same
 * arguments, tests after its conservative culling (a box culled for a 32 x 32
 * tile is not tested for any pixel of it), into *live_pairs (host). Renders
 * nothing; synchronises the context's stream. This is the work a launch
 * performs, against which its ALU fraction is stated. Errors as
 * ag_render_depth; AG_ERR_INVALID for a NULL live_pairs. */
ag_status ag_depth_live_pairs(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                              const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams,
                              uint64_t* live_pairs);

#ifdef __cplusplus
}
#endif

#endif /* AG_MEASURE_H */
