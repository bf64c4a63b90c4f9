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

constexpr int kTaskBlock = 64;  // measured over 32 .. 256: 64 is best by about 1 %
constexpr int kObs = 13;

__device__ __forceinline__ float norm3(float x, float y, float z) { return sqrtf(fmaf(z, z, fmaf(y, y, x * x))); }

__device__ __forceinline__ V3 load_goal(const ReachArgs& a, uint32_t i) {
  const uint32_t n = a.fb.n;
  return {a.goals[i], a.goals[n + i], a.goals[2 * n + i]};
}

// obs = (p - g, v, q with w >= 0, Omega)
__device__ __forceinline__ void observe(const VState& s, V3 g, float* o) {
  const float sgn = s.q.w < 0.f ? -1.f : 1.f;
  o[0] = s.p.x - g.x; o[1] = s.p.y - g.y; o[2] = s.p.z - g.z;
  o[3] = s.v.x; o[4] = s.v.y; o[5] = s.v.z;
  o[6] = sgn * s.q.w; o[7] = sgn * s.q.x; o[8] = sgn * s.q.y; o[9] = sgn * s.q.z;
  o[10] = s.w.x; o[11] = s.w.y; o[12] = s.w.z;
}

// Boxes of environment env read two at a time from the env-ordered array
// (plain loads: a re-draw in the same launch rewrites them).
struct EnvBoxPairs {
  const float* boxes;
  uint32_t n, env;
  __device__ __forceinline__ float2 at(int j, int f, int n_obs) const {
    const int k0 = 2 * j, k1 = 2 * j + 1;
    return make_float2(staged_field(f, boxes[((size_t)k0 * 10 + f) * n + env]),
                       staged_field(f, k1 < n_obs ? boxes[((size_t)k1 * 10 + f) * n + env] : box_pad_field(f)));
  }
  __device__ __forceinline__ bool any_hit_min(V3 p, float r2, int n_obs, float& m) const {
    const float2 px = dup2(p.x), py = dup2(p.y), pz = dup2(p.z);
    bool hit = false;
    m = __int_as_float(0x7f800000);
    for (int j = 0; j < (n_obs + 1) >> 1; ++j)
      hit |= pair_hits_min(px, py, pz, r2, at(j, 0, n_obs), at(j, 1, n_obs), at(j, 2, n_obs), at(j, 3, n_obs),
                           at(j, 4, n_obs), at(j, 5, n_obs), at(j, 6, n_obs), at(j, 7, n_obs), at(j, 8, n_obs),
                           at(j, 9, n_obs), m);
    return hit;
  }
  __device__ __forceinline__ NoBoxes staged() const { return {}; }
  __device__ __forceinline__ void reload(const FleetBuffers&, uint32_t) {}
};

// Reward, termination and in-place reset of environment i after its step
// (s: its state after the step; hit: it collided, and the step already
// re-drew it), then its observation into o[0..12].
__device__ __forceinline__ void reach_tail(const ReachArgs& a, uint32_t i, VState s, bool hit, uint32_t steps_before,
                                           V3 g, float* o) {
  const uint32_t steps = steps_before + 1u;
  const float dist = norm3(s.p.x - g.x, s.p.y - g.y, s.p.z - g.z);
  const float speed = norm3(s.v.x, s.v.y, s.v.z);
  const float rate = norm3(s.w.x, s.w.y, s.w.z);
  const bool end = hit || dist > a.max_dist || steps >= a.max_steps;
  a.reward[i] = hit ? -a.crash : -fmaf(a.w_omega, rate, fmaf(a.w_v, speed, dist));
  a.done[i] = end ? 1 : 0;
  a.steps[i] = end ? 0u : steps;
  if (end && !hit) {
    reset_env(a.fb, i, a.seed_lo, a.seed_hi);
    s = load_state(a.fb.state, a.fb.n, i);
  }
  observe(s, g, o);
}

// Coalesced write of the staged [kTaskBlock][13] observation rows, warp by
// warp: the rows of a warp's 32 environments are one contiguous slice of the
// stage and of obs, so each warp writes its own after a __syncwarp and no
// warp waits for the rest of the block.
__device__ __forceinline__ void write_obs(const ReachArgs& a, const float* stage) {
  __syncwarp();
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const size_t base = ((size_t)blockIdx.x * kTaskBlock + warp * 32u) * kObs;
  const size_t total = (size_t)a.fb.n * kObs;
  const float* ws = stage + warp * 32u * kObs;
#pragma unroll
  for (uint32_t t = lane; t < 32u * kObs; t += 32u)
    if (base + t < total) a.obs[base + t] = ws[t];
}

// One task step of environment i = thread: actions -> commands, one fleet
// step (controller, allocation, integration, collision test and reset, as in
// the fused fleet step), then reach_tail. Every environment shares the task's
// command mode, so warps are mode-uniform without a grouping permutation.
// Without boxes the step is memory-latency bound: a bound of 14 blocks (28
// warps) per SM measured best, against 16 blocks (64 registers, more spills)
// and 20 (48 registers). With boxes it keeps 12 warps per SM (170 registers).
template <int INTEG, bool DRAG, bool BOXES>
__global__ void __launch_bounds__(kTaskBlock, BOXES ? 384 / kTaskBlock : 896 / kTaskBlock)
    k_reach_step(ReachArgs a, StepParams P, int substeps) {
  __shared__ float stage[kTaskBlock * kObs];  // odd row length: conflict-free
  const FleetBuffers& fb = a.fb;
  const uint32_t i = blockIdx.x * kTaskBlock + threadIdx.x;
  const uint32_t n = fb.n;
  uint32_t resets = 0, tests = 0;
  if (i < n) {
    // everything the step reads from memory, requested up front
    const float4 act = reinterpret_cast<const float4*>(a.actions)[i];
    const V3 g = load_goal(a, i);
    const uint32_t steps_before = a.steps[i];
    const float v[4] = {act.x, act.y, act.z, act.w};
    float t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = fmaf(a.scale[k], fminf(fmaxf(v[k], -1.f), 1.f), a.offset[k]);
    const Command cm = prepare_command(fb.modes[i], t[0], t[1], t[2], t[3]);
    const int nrot = rotor_count(fb, i);
    // environment i's place in the slot-ordered box copy (a re-draw updates it there)
    const uint32_t slot = fb.slot_of ? fb.slot_of[i] : i;
    const int n_obs = (int)fb.n_obs;
    bool hit = false;
    VState s;
    if (BOXES) {
      EnvBoxPairs bx{fb.boxes, n, i};
      if (nrot == 4)
        s = simulate_cmd<4, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit, tests);
      else if (nrot == 6)
        s = simulate_cmd<6, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit, tests);
      else
        s = simulate_cmd<8, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, n_obs, bx, a.seed_lo, a.seed_hi, resets, hit, tests);
    } else {
      NoBoxSource none;
      if (nrot == 4)
        s = simulate_cmd<4, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit, tests);
      else if (nrot == 6)
        s = simulate_cmd<6, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit, tests);
      else
        s = simulate_cmd<8, INTEG, DRAG>(fb, P, i, slot, cm, 1, substeps, 0, none, a.seed_lo, a.seed_hi, resets, hit, tests);
    }
    fb.collided[i] = hit ? 1 : 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) fb.targets[k * n + i] = t[k];  // the commands, as ag_set_commands keeps them
    reach_tail(a, i, s, hit, steps_before, g, stage + threadIdx.x * kObs);
  }
  write_obs(a, stage);
}

__global__ void __launch_bounds__(kTaskBlock) k_reach_observe(ReachArgs a) {
  __shared__ float stage[kTaskBlock * kObs];
  const uint32_t i = blockIdx.x * kTaskBlock + threadIdx.x;
  if (i < a.fb.n) observe(load_state(a.fb.state, a.fb.n, i), load_goal(a, i), stage + threadIdx.x * kObs);
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
