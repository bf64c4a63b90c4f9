// task.cu — the reach-a-setpoint task around the fleet step.
//
// The paper trains policies that fly a multirotor to a goal setpoint through
// the attitude or the velocity command interface (Sec. I). One task step is
// the policy's actions mapped to the commands of every environment, one fleet
// step (ag_step), then one pass per environment that scores the step,
// decides whether the episode ended, re-draws the environments whose episode
// ended without a collision (a collision already re-drew its environment
// inside the step) and writes the observation of the state the policy sees
// next:
//   obs    = (p - g, v, q with w >= 0, Omega)                       [n][13]
//   reward = -crash after a collision, else -|p - g| - w_v |v| - w_omega |Omega|
//   done   = collided or |p - g| > max_dist or steps >= max_steps
#include <cstdint>

#include <cuda_runtime.h>

#include "fleet_sim.cuh"
#include "task_internal.h"

namespace agk {
namespace {

constexpr int kTaskBlock = 128;
constexpr int kObs = 13;

__global__ void __launch_bounds__(256) k_reach_actions(ReachArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = a.fb.n;
  if (i >= n) return;
  const float4 act = reinterpret_cast<const float4*>(a.actions)[i];
  const float v[4] = {act.x, act.y, act.z, act.w};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    a.fb.targets[k * n + i] = fmaf(a.scale[k], fminf(fmaxf(v[k], -1.f), 1.f), a.offset[k]);
}

__device__ __forceinline__ float norm3(float x, float y, float z) { return sqrtf(x * x + y * y + z * z); }

__global__ void __launch_bounds__(kTaskBlock) k_reach_tail(ReachArgs a, bool observe_only) {
  __shared__ float stage[kTaskBlock * kObs];  // odd row length: conflict-free
  const uint32_t i = blockIdx.x * kTaskBlock + threadIdx.x;
  const uint32_t n = a.fb.n;
  if (i < n) {
    const float* st = a.fb.state;
    if (!observe_only) {
      const bool hit = a.fb.collided[i] != 0;
      const uint32_t steps = a.steps[i] + 1u;
      const float ex = st[0 * n + i] - a.goals[0 * n + i], ey = st[1 * n + i] - a.goals[1 * n + i],
                  ez = st[2 * n + i] - a.goals[2 * n + i];
      const float dist = norm3(ex, ey, ez);
      const float speed = norm3(st[3 * n + i], st[4 * n + i], st[5 * n + i]);
      const float rate = norm3(st[10 * n + i], st[11 * n + i], st[12 * n + i]);
      const bool end = hit || dist > a.max_dist || steps >= a.max_steps;
      a.reward[i] = hit ? -a.crash : -(dist + a.w_v * speed + a.w_omega * rate);
      a.done[i] = end ? 1 : 0;
      a.steps[i] = end ? 0u : steps;
      if (end && !hit) reset_env(a.fb, i, a.seed_lo, a.seed_hi);
    }
    const float sgn = st[6 * n + i] < 0.f ? -1.f : 1.f;
    float* o = stage + threadIdx.x * kObs;
    o[0] = st[0 * n + i] - a.goals[0 * n + i];
    o[1] = st[1 * n + i] - a.goals[1 * n + i];
    o[2] = st[2 * n + i] - a.goals[2 * n + i];
#pragma unroll
    for (int r = 3; r < 6; ++r) o[r] = st[r * n + i];
#pragma unroll
    for (int r = 6; r < 10; ++r) o[r] = sgn * st[r * n + i];
#pragma unroll
    for (int r = 10; r < 13; ++r) o[r] = st[r * n + i];
  }
  __syncthreads();
  // coalesced write of the block's [kTaskBlock][13] rows
  const size_t base = (size_t)blockIdx.x * kTaskBlock * kObs;
  const size_t total = (size_t)n * kObs;
  for (int t = threadIdx.x; t < kTaskBlock * kObs; t += kTaskBlock)
    if (base + t < total) a.obs[base + t] = stage[t];
}

}  // namespace

cudaError_t launch_reach_actions(const ReachArgs& a, cudaStream_t st) {
  k_reach_actions<<<(a.fb.n + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reach_tail(const ReachArgs& a, bool observe_only, cudaStream_t st) {
  k_reach_tail<<<(a.fb.n + kTaskBlock - 1) / kTaskBlock, kTaskBlock, 0, st>>>(a, observe_only);
  return cudaGetLastError();
}

}  // namespace agk
