// fleet_internal.h — launch interface between the C-ABI layer and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ag.h"
#include "fleet_device.cuh"
#include "reset_sampler.cuh"

namespace agk {

// NVTX range over a host-side span (a C-ABI call's checks and enqueueing, a
// serving chunk), so a profiler's timeline names what issued each kernel.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device buffers of one fleet (all structure-of-arrays over n environments).
struct FleetBuffers {
  float* state;        // [13][n]  p, v, q, Omega
  float* motors;       // [8][n]   rotor thrusts
  float* body;         // [4][n]   m, Jxx, Jyy, Jzz
  uint8_t* modes;      // [n]
  float* targets;      // [4][n]
  float* boxes;        // [n_obs][10][n]
  uint32_t* epoch;     // [n]
  uint8_t* collided;   // [n]     hit a box during the last call
  uint32_t* reset_ids; // [n]     compact list of envs reset during the last call
  uint32_t* n_reset;   // [1]     length of that list
  // scratch of the unfused path (one launch per stage)
  float* cmd;          // [4][n]  commanded wrench
  float* wrench;       // [4][n]  realised wrench
  uint32_t* resets;    // [n]     resets of this call per env
  uint8_t* hits;       // [n]     collision of the current step
  uint32_t* order;     // [n]     thread slot -> env, grouped by rotor type and mode (NULL = identity)
  float2* boxes_slot;  // [ceil(n_obs/2)][10][n] the boxes in slot order, in pairs: element
                       // (j*10 + f)*n + i = (field f of box 2j, of box 2j+1) of env order[i],
                       // in the staged form of staged_field (-c, -h, -w, 2u)
  uint32_t* slot_of;   // [n]     inverse of order (NULL when no obstacle re-draw is needed)
  const BoxRandDev* box_rand;  // [n_obs] obstacle re-draw on reset (NULL = boxes keep their poses)
  unsigned long long* tests_run;  // [1] exact collision tests of the last fused call (NULL = not counted)
  uint32_t n, n_quad, n_hexa, n_octo, n_obs;
};

// Launch constants of a configuration: gains, FP64-computed allocation
// matrices of the three rotor types, substep length, motor-lag factor,
// drag, squared collision radius, thrust limit and the reset key.
StepParams step_params_for(const ag_config& c, uint64_t seed);

// Launches return cudaGetLastError() of their launch.
cudaError_t launch_fused_step(const FleetBuffers& fb, const StepParams& P, int integrator, int n_steps,
                              int substeps, cudaStream_t st);
cudaError_t launch_reset(const FleetBuffers& fb, const uint8_t* mask, uint32_t seed_lo, uint32_t seed_hi,
                         cudaStream_t st);
// The controller alone: fb.cmd[4][n] = commanded (f, M) of every environment
// at fb.state (the unfused path's controller stage).
cudaError_t launch_controller(const FleetBuffers& fb, const StepParams& P, cudaStream_t st);
cudaError_t launch_plain_step(const FleetBuffers& fb, const StepParams& P, int integrator, int n_steps,
                              int substeps, cudaStream_t st);

// Builds fb.order from the current modes and rotor types (one launch; scratch
// holds order_scratch_words(n) words), then refreshes fb.boxes_slot.
cudaError_t launch_build_order(const FleetBuffers& fb, uint32_t* scratch, cudaStream_t st);
size_t order_scratch_words(uint32_t n);
// Elements (float2) of fb.boxes_slot for n envs with n_obs boxes each.
inline size_t box_pair_elems(size_t n, size_t n_obs) { return (n_obs + 1) / 2 * 10 * n; }

// Refreshes fb.boxes_slot from fb.boxes and fb.order (after the boxes change).
// An odd box count is padded with a box at 1e30 that no sphere can touch.
cudaError_t launch_permute_boxes(const FleetBuffers& fb, cudaStream_t st);

// Dynamic shared memory of a fused-kernel block of B threads: box pairs 1..
// of every thread (pair 0 stays in registers).
inline size_t fused_smem_bytes(int n_obs, int B) {
  const int pairs = (n_obs + 1) / 2;
  return pairs > 1 ? (size_t)(pairs - 1) * 10 * B * 8 : 0;
}

// Launch choices of the fused kernel. Defaults: mode-grouped order, the
// block size (from 64, 128, 96, 32) with the most resident warps per SM by
// the occupancy calculator (block = 0 here), and collision tests skipped
// while a vehicle provably cannot reach a box. Tuning overrides (read at each
// launch): AG_FUSED_ORDER=identity runs env i in slot i (the ungrouped
// ablation), AG_FUSED_BLOCK=32..128 (multiple of 32) sets the block size,
// AG_FUSED_SKIP=0 runs the exact test at every step (same results, the
// reference the skip is checked against).
struct FusedTuning { bool sorted; int block; bool skip; };
FusedTuning fused_tuning_from_env(int n_obs);

}  // namespace agk
