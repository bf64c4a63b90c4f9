// task_internal.h — launch interface of the reach-a-setpoint task kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fleet_internal.h"

namespace agk {

struct ReachArgs {
  FleetBuffers fb;
  const float* actions;  // [n][4], 16-byte aligned
  const float* goals;    // [3][n]
  uint32_t* steps;       // [n] steps taken in the current episode
  float* obs;            // [n][13]
  float* reward;         // [n]
  uint8_t* done;         // [n]
  float scale[4], offset[4];
  float w_v, w_omega, crash, max_dist;
  uint32_t max_steps;
  uint32_t seed_lo, seed_hi;
};

// One task step in one launch: commands = offset + scale * clamp(actions,
// -1, 1) into fb.targets, one fleet step of `substeps` substeps (collided
// flags set; the reset list is left alone, the done flags carry the episode
// ends), reward and termination, in-place reset of the episodes that ended
// without a collision, observations of the new state.
cudaError_t launch_reach_step(const ReachArgs& a, const StepParams& P, int integrator, int substeps, cudaStream_t st);
// Observations of the current states alone.
cudaError_t launch_reach_observe(const ReachArgs& a, cudaStream_t st);

}  // namespace agk
