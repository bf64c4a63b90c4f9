// depth_internal.h — launch interface of the depth ray caster.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fleet_device.cuh"

namespace agk {

struct DepthArgs {
  const float* state;      // [13][n]
  const float* boxes;      // [n_obs][10][n]
  const uint32_t* env_ids; // [n_cams] or NULL (camera j = env j)
  float* out;              // [n_cams][height][width]
  uint32_t n, n_obs, n_cams, width, height;
  uint32_t cam0;           // first camera of a launch (set by the launcher)
  float inv_f;             // tan(hfov / 2) / (width / 2)
  float max_range;
  float offset[3];         // camera position in the body frame
  int vec_store;           // set by the launcher: width % 4 == 0 and out 16-byte aligned (one float4 per row)
  // Measurement variants (ag_measure.h); both 0 / NULL for ag_render_depth.
  int ieee_div;                    // 1: correctly rounded reciprocals instead of the fast approximation
  unsigned long long* live_pairs;  // non-NULL: count the (pixel, box) pairs left after culling, render nothing
};

cudaError_t launch_render_depth(const DepthArgs& a, cudaStream_t st);

}  // namespace agk
