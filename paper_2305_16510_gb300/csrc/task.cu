// task.cu — the reach-a-setpoint task around the fleet step.
//
// The paper trains policies that fly a multirotor to a goal setpoint through
// the attitude or the velocity command interface (Sec. I). One task step is
// one kernel launch: per environment the policy's action becomes its command,
// the fleet step runs (the fused step's per-vehicle loop: controller,
// allocation, integration, collision test and reset), and the step is scored;
// an episode that ended without a collision is re-drawn in place (a collision
// already re-drew its environment inside the step), and the observation of
// the state the policy sees next is written:
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

__device__ __forceinline__ float norm3(float x, float y, float z) { return sqrtf(x * x + y * y + z * z); }

// Boxes of environment env read two at a time from the env-ordered array
// (plain loads: a re-draw in the same launch rewrites them).
struct EnvBoxPairs {
  const float* boxes;
  uint32_t n, env;
  __device__ __forceinline__ float2 at(int j, int f, int n_obs) const {
    const int k0 = 2 * j, k1 = 2 * j + 1;
    return make_float2(boxes[((size_t)k0 * 10 + f) * n + env],
                       k1 < n_obs ? boxes[((size_t)k1 * 10 + f) * n + env] : box_pad_field(f));
  }
  __device__ __forceinline__ bool any_hit(V3 p, float r2, int n_obs) const {
    const float2 px = dup2(p.x), py = dup2(p.y), pz = dup2(p.z);
    bool hit = false;
    for (int j = 0; j < (n_obs + 1) >> 1; ++j)
      hit |= pair_hits(px, py, pz, r2, at(j, 0, n_obs), at(j, 1, n_obs), at(j, 2, n_obs), at(j, 3, n_obs),
                       at(j, 4, n_obs), at(j, 5, n_obs), at(j, 6, n_obs), at(j, 7, n_obs), at(j, 8, n_obs),
                       at(j, 9, n_obs));
    return hit;
  }
  __device__ __forceinline__ NoBoxes staged() const { return {}; }
  __device__ __forceinline__ void reload(const FleetBuffers&, uint32_t) {}
};

// Reward, termination and in-place reset of environment i after its step
// (hit: it collided, and the step already re-drew it), then its observation
// into o[0..12].
__device__ __forceinline__ void reach_tail(const ReachArgs& a, uint32_t i, bool hit, bool observe_only, float* o) {
  const uint32_t n = a.fb.n;
  const float* st = a.fb.state;
  if (!observe_only) {
    const uint32_t steps = a.steps[i] + 1u;
    const float dist = norm3(st[0 * n + i] - a.goals[0 * n + i], st[1 * n + i] - a.goals[1 * n + i],
                             st[2 * n + i] - a.goals[2 * n + i]);
    const float speed = norm3(st[3 * n + i], st[4 * n + i], st[5 * n + i]);
    const float rate = norm3(st[10 * n + i], st[11 * n + i], st[12 * n + i]);
    const bool end = hit || dist > a.max_dist || steps >= a.max_steps;
    a.reward[i] = hit ? -a.crash : -(dist + a.w_v * speed + a.w_omega * rate);
    a.done[i] = end ? 1 : 0;
    a.steps[i] = end ? 0u : steps;
    if (end && !hit) reset_env(a.fb, i, a.seed_lo, a.seed_hi);
  }
  const float sgn = st[6 * n + i] < 0.f ? -1.f : 1.f;
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

// Coalesced write of the block's staged [kTaskBlock][13] observation rows.
__device__ __forceinline__ void write_obs(const ReachArgs& a, const float* stage) {
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kTaskBlock * kObs;
  const size_t total = (size_t)a.fb.n * kObs;
  for (int t = threadIdx.x; t < kTaskBlock * kObs; t += kTaskBlock)
    if (base + t < total) a.obs[base + t] = stage[t];
}

// One task step of environment i = thread: actions -> commands, one fleet
// step (controller, allocation, integration, collision test and reset, as in
// the fused fleet step), then reach_tail. Every environment shares the task's
// command mode, so warps are mode-uniform without a grouping permutation.
template <int INTEG, bool DRAG, bool BOXES>
__global__ void __launch_bounds__(kTaskBlock, BOXES ? 3 : 4) k_reach_step(ReachArgs a, StepParams P, int substeps) {
  __shared__ float stage[kTaskBlock * kObs];  // odd row length: conflict-free
  const FleetBuffers& fb = a.fb;
  const uint32_t i = blockIdx.x * kTaskBlock + threadIdx.x;
  const uint32_t n = fb.n;
  uint32_t resets = 0;
  if (i < n) {
    const float4 act = reinterpret_cast<const float4*>(a.actions)[i];
    const float v[4] = {act.x, act.y, act.z, act.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) fb.targets[k * n + i] = fmaf(a.scale[k], fminf(fmaxf(v[k], -1.f), 1.f), a.offset[k]);
    const int nrot = rotor_count(fb, i);
    const int n_obs = (int)fb.n_obs;
    bool hit = false;
    if (BOXES) {
      EnvBoxPairs bx{fb.boxes, n, i};
      if (nrot == 4) simulate<4, INTEG, DRAG>(fb, P, i, i, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit);
      else if (nrot == 6) simulate<6, INTEG, DRAG>(fb, P, i, i, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit);
      else simulate<8, INTEG, DRAG>(fb, P, i, i, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit);
    } else {
      NoBoxSource none;
      if (nrot == 4) simulate<4, INTEG, DRAG>(fb, P, i, i, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit);
      else if (nrot == 6) simulate<6, INTEG, DRAG>(fb, P, i, i, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit);
      else simulate<8, INTEG, DRAG>(fb, P, i, i, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit);
    }
    fb.collided[i] = hit ? 1 : 0;
    reach_tail(a, i, hit, false, stage + threadIdx.x * kObs);
  }
  append_compact(resets > 0u, i, fb.reset_ids, fb.n_reset);
  write_obs(a, stage);
}

__global__ void __launch_bounds__(kTaskBlock) k_reach_observe(ReachArgs a) {
  __shared__ float stage[kTaskBlock * kObs];
  const uint32_t i = blockIdx.x * kTaskBlock + threadIdx.x;
  if (i < a.fb.n) reach_tail(a, i, false, true, stage + threadIdx.x * kObs);
  write_obs(a, stage);
}

template <int INTEG, bool DRAG>
cudaError_t launch_step_t(const ReachArgs& a, const StepParams& P, int substeps, cudaStream_t st) {
  const unsigned grid = (a.fb.n + kTaskBlock - 1) / kTaskBlock;
  if (a.fb.n_obs > 0)
    k_reach_step<INTEG, DRAG, true><<<grid, kTaskBlock, 0, st>>>(a, P, substeps);
  else
    k_reach_step<INTEG, DRAG, false><<<grid, kTaskBlock, 0, st>>>(a, P, substeps);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reach_step(const ReachArgs& a, const StepParams& P, int integrator, int substeps, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.fb.n_reset, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const bool drag = P.drag != 0.f;
  if (integrator == kIntegRK4)
    return drag ? launch_step_t<kIntegRK4, true>(a, P, substeps, st) : launch_step_t<kIntegRK4, false>(a, P, substeps, st);
  return drag ? launch_step_t<kIntegSIE, true>(a, P, substeps, st) : launch_step_t<kIntegSIE, false>(a, P, substeps, st);
}

cudaError_t launch_reach_observe(const ReachArgs& a, cudaStream_t st) {
  k_reach_observe<<<(a.fb.n + kTaskBlock - 1) / kTaskBlock, kTaskBlock, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace agk
