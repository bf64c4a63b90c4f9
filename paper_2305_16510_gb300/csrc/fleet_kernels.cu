// fleet_kernels.cu — the fused fleet-step kernel, the reset kernel and the
// unfused (one launch per stage) comparison path.
//
// Fused step (the hot path): one thread owns one environment for a whole
// launch of n_steps steps. Its 13 state words, motor thrusts, body
// parameters and command live in registers across every substep; its boxes
// are read only when a collision test runs (the first step, then only while
// the vehicle may be within reach of a box), as coalesced rows of the
// slot-ordered pair copy; state and command are read at the start and
// written at the end of the launch (coalesced structure-of-arrays rows).
// Collision resets happen in registers; the reset list is built with one
// __ballot_sync + __popc prefix and one atomicAdd per warp.
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

#include "fleet_internal.h"
#include "fleet_sim.cuh"
#include "reset_sampler.cuh"

namespace agk {
namespace {

// Dynamic shared memory cap of the fused kernel (box staging).
constexpr size_t kFusedSmemCap = 200 * 1024;

// Tuning override (read at each launch): AG_FUSED_BOXES=smem stages every
// thread's boxes on chip for the whole launch instead of reading them from
// the global pair copy when a collision test runs (the ablation of that
// choice; results are identical).
bool fused_boxes_staged_from_env() {
  const char* v = std::getenv("AG_FUSED_BOXES");
  return v && std::strcmp(v, "smem") == 0;
}

// Where a launch's collision tests read the boxes from.
enum : int {
  kBoxesNone = 0,    // no obstacles
  kBoxesStaged = 1,  // staged per thread: pair 0 in registers, the others in shared memory
  kBoxesGlobal = 2,  // the slot-ordered pair copy in global memory, read when a test runs
};

// Thread slot i of the launch simulates environment order[i] (a permutation
// that groups environments of equal rotor count and command mode, so the
// mode branches of the controller are warp-uniform), or environment i when
// order is NULL. A collision test that cannot hit is skipped (simulate_cmd),
// so tests are rare after the first step; by default a test reads the
// environment's box pairs from the slot-ordered copy in global memory, which
// needs no shared memory. Threads of one command mode run the loop
// compiled for that mode (simulate). The bound of 4 blocks of 128 threads
// per SM holds the kernel under 128 registers, 4 warps per SM sub-partition
// (16 per SM); a bound of 3 (140 registers, 12 warps per SM) measured
// slower. The staged form keeps each thread's boxes on chip for the launch
// instead: boxes 0 and 1 in registers, the others in shared memory
// as float4 [pair][field pair][thread], so a warp's 16-byte loads of two
// fields are consecutive and conflict-free (a thread reads only what it
// wrote, so no barrier is needed).
// Without obstacles the kernel stays within 128 registers. A quad-only
// semi-implicit-Euler fleet without obstacles needs about 70 (no spills),
// and its bound of 7 blocks per SM lets a 131,072-vehicle fleet run in one
// wave; fleets with hexa and octo rotors keep the looser bound, which
// measured faster for them.
template <int INTEG, bool QUAD_ONLY, bool DRAG, int BOXES>
__global__ void __launch_bounds__(128, BOXES == kBoxesGlobal ? 4
                                       : (BOXES == kBoxesStaged ? 3 : ((QUAD_ONLY && INTEG == kIntegSIE) ? 7 : 4)))
    k_fused_step(FleetBuffers fb, StepParams P, int n_steps, int substeps) {
  extern __shared__ float4 sm_pairs[];  // [ceil(n_obs / 2) - 1][5][blockDim.x] box pairs 1..
  const int B = blockDim.x;
  const uint32_t slot = blockIdx.x * B + threadIdx.x;
  const bool active = slot < fb.n;
  const uint32_t env = active ? (fb.order ? fb.order[slot] : slot) : slot;
  RegSmemBoxPairs bx;
  bx.sm = sm_pairs + threadIdx.x;
  bx.B = B;
#pragma unroll
  for (int f = 0; f < 10; ++f) bx.r[f] = make_float2(0.f, 0.f);
  const int n_obs = (int)fb.n_obs;
  if (BOXES == kBoxesStaged && active && n_obs > 0) {
    const int pairs = (n_obs + 1) / 2;
    if (fb.order) {
      // the slot-ordered pair copy: coalesced 8-byte rows
#pragma unroll
      for (int f = 0; f < 10; ++f) bx.r[f] = fb.boxes_slot[(size_t)f * fb.n + slot];
      for (int r = 10; r < pairs * 10; r += 2) {
        const float2 lo = fb.boxes_slot[(size_t)r * fb.n + slot], hi = fb.boxes_slot[(size_t)(r + 1) * fb.n + slot];
        bx.sm[(r - 10) / 2 * B] = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
    } else {
      // ungrouped (env == slot): pair up the env-ordered rows here
      bx.reload(fb, slot);
      for (int j = 1; j < pairs; ++j) {
        const int k0 = 2 * j, k1 = 2 * j + 1;
#pragma unroll
        for (int f = 0; f < 10; f += 2) {
          float v[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {  // a_f, b_f, a_f+1, b_f+1
            const int k = (c & 1) ? k1 : k0, ff = f + (c >> 1);
            const float raw = k < n_obs ? fb.boxes[((size_t)k * 10 + ff) * fb.n + slot] : box_pad_field(ff);
            v[c] = staged_field(ff, raw);
          }
          bx.sm[((j - 1) * 5 + f / 2) * B] = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
    }
  }
  uint32_t resets = 0, tests = 0;
  bool any_hit = false;
  if (active) {
    const int nrot = QUAD_ONLY ? 4 : rotor_count(fb, env);
    if (BOXES == kBoxesGlobal) {
      GlobalBoxPairs gx{fb.boxes_slot, fb.n, slot};
      if (nrot == 4)
        simulate<4, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, gx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else if (nrot == 6)
        simulate<6, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, gx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else
        simulate<8, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, gx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
    } else if (BOXES == kBoxesStaged) {
      if (nrot == 4)
        simulate<4, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, bx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else if (nrot == 6)
        simulate<6, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, bx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else
        simulate<8, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, n_obs, bx, P.seed_lo, P.seed_hi, resets, any_hit, tests);
    } else {
      NoBoxSource none;
      if (nrot == 4)
        simulate<4, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, 0, none, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else if (nrot == 6)
        simulate<6, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, 0, none, P.seed_lo, P.seed_hi, resets, any_hit, tests);
      else
        simulate<8, INTEG, DRAG, true>(fb, P, env, slot, n_steps, substeps, 0, none, P.seed_lo, P.seed_hi, resets, any_hit, tests);
    }
    fb.collided[env] = any_hit ? 1 : 0;
  }
  append_compact(resets > 0u, env, fb.reset_ids, fb.n_reset);
  if (BOXES != kBoxesNone && fb.tests_run) {  // one atomic per warp
    const unsigned t = __reduce_add_sync(0xFFFFFFFFu, tests);
    if ((threadIdx.x & 31u) == 0u && t) atomicAdd(fb.tests_run, (unsigned long long)t);
  }
}

// Grouping permutation: key = rotor-type index * 4 + mode (12 keys). Slots
// [w * W, (w + 1) * W), W = 4,096, hold the environments of the same window, stably
// partitioned by key: inside a window the controller's mode branches become
// warp-uniform (at most one mixed warp per key boundary), and since a window's
// envs are loaded by blocks that run at the same time, the sectors their
// gathers share are served from L2 instead of being fetched again from DRAM.
// One block per window: the key totals give each key's start; then, 1,024
// envs at a time, each env is ranked inside its warp with __match_any_sync and
// offset by its key's running position and the preceding warps' counts.
constexpr int kOrderThreads = 1024;
constexpr int kOrderSub = 4;                                  // sub-windows per window
constexpr int kOrderWindow = kOrderThreads * kOrderSub;       // 4,096 envs

__device__ __forceinline__ uint32_t order_key(const FleetBuffers& fb, uint32_t i) {
  const int nrot = rotor_count(fb, i);
  const uint32_t m = fb.modes[i] > 3 ? 3u : fb.modes[i];
  return (uint32_t)(nrot == 4 ? 0 : (nrot == 6 ? 1 : 2)) * 4u + m;
}

__global__ void __launch_bounds__(kOrderThreads) k_order_window(FleetBuffers fb) {
  __shared__ uint32_t warp_count[kOrderThreads / 32][12];
  __shared__ uint32_t key_next[12];  // next free position of each key in the window
  const uint32_t base = blockIdx.x * kOrderWindow;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // pass 1: totals per key over the window -> start position of each key
  if (threadIdx.x < 12) key_next[threadIdx.x] = 0;
  __syncthreads();
  for (int sub = 0; sub < kOrderSub; ++sub) {
    const uint32_t i = base + sub * kOrderThreads + threadIdx.x;
    if (i < fb.n) atomicAdd(&key_next[order_key(fb, i)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < 12; ++k) {
      const uint32_t c = key_next[k];
      key_next[k] = run;
      run += c;
    }
  }
  __syncthreads();
  // pass 2: sub-window by sub-window, stable ranks inside each key
  for (int sub = 0; sub < kOrderSub; ++sub) {
    const uint32_t i = base + sub * kOrderThreads + threadIdx.x;
    const bool active = i < fb.n;
    const uint32_t key = active ? order_key(fb, i) : 12u;
    const unsigned same = __match_any_sync(0xFFFFFFFFu, key);
    const uint32_t rank = __popc(same & ((1u << lane) - 1u));
    if (lane < 12) warp_count[warp][lane] = 0;
    __syncwarp();
    if (active && rank == 0) warp_count[warp][key] = __popc(same);
    __syncthreads();
    if (active) {
      uint32_t pos = key_next[key] + rank;
      for (int w = 0; w < warp; ++w) pos += warp_count[w][key];
      fb.order[base + pos] = i;
      if (fb.slot_of) fb.slot_of[i] = base + pos;
    }
    __syncthreads();
    if (threadIdx.x < 12) {  // advance each key by its count in this sub-window
      uint32_t c = 0;
      for (int w = 0; w < kOrderThreads / 32; ++w) c += warp_count[w][threadIdx.x];
      key_next[threadIdx.x] += c;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_permute_boxes(FleetBuffers fb) {
  const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= fb.n) return;
  const uint32_t env = fb.order[slot];
  const int n_obs = (int)fb.n_obs;
  for (int j = 0; j < (n_obs + 1) / 2; ++j) {
    const int k0 = 2 * j, k1 = 2 * j + 1;
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      const float a = fb.boxes[((size_t)k0 * 10 + f) * fb.n + env];
      const float b = k1 < n_obs ? fb.boxes[((size_t)k1 * 10 + f) * fb.n + env] : box_pad_field(f);
      fb.boxes_slot[(size_t)(j * 10 + f) * fb.n + slot] = make_float2(staged_field(f, a), staged_field(f, b));
    }
  }
}

// ag_reset: resample masked environments, clear collided flags, list them.
__global__ void __launch_bounds__(256) k_reset(FleetBuffers fb, const uint8_t* mask, uint32_t seed_lo,
                                               uint32_t seed_hi) {
  const uint32_t env = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = fb.n;
  const bool active = env < n;
  const bool flag = active && (mask == nullptr || mask[env] != 0);
  if (flag) reset_env(fb, env, seed_lo, seed_hi);
  if (active) fb.collided[env] = 0;
  append_compact(flag, env, fb.reset_ids, fb.n_reset);
}

// ------------------------------------------------ unfused comparison path --
__global__ void __launch_bounds__(256) k_plain_controller(FleetBuffers fb, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fb.n) return;
  const uint32_t n = fb.n;
  VState s = load_state(fb.state, n, i);
  normalize(s.q);
  V3 b3;
  Wrench4 c = controller(s, load_command(fb, i), load_body(fb.body, n, i), P, b3);
  fb.cmd[0 * n + i] = c.f; fb.cmd[1 * n + i] = c.mx; fb.cmd[2 * n + i] = c.my; fb.cmd[3 * n + i] = c.mz;
}

template <int NROT>
__device__ __forceinline__ void plain_allocate_one(const FleetBuffers& fb, const StepParams& P, uint32_t i) {
  const uint32_t n = fb.n;
  float u[NROT];
#pragma unroll
  for (int k = 0; k < NROT; ++k) u[k] = fb.motors[k * n + i];
  Wrench4 c = {fb.cmd[0 * n + i], fb.cmd[1 * n + i], fb.cmd[2 * n + i], fb.cmd[3 * n + i]};
  Wrench4 W = allocate<NROT>(c, u, P);
#pragma unroll
  for (int k = 0; k < NROT; ++k) fb.motors[k * n + i] = u[k];
  fb.wrench[0 * n + i] = W.f; fb.wrench[1 * n + i] = W.mx; fb.wrench[2 * n + i] = W.my; fb.wrench[3 * n + i] = W.mz;
}

__global__ void __launch_bounds__(256) k_plain_allocate(FleetBuffers fb, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fb.n) return;
  const int nrot = rotor_count(fb, i);
  if (nrot == 4) plain_allocate_one<4>(fb, P, i);
  else if (nrot == 6) plain_allocate_one<6>(fb, P, i);
  else plain_allocate_one<8>(fb, P, i);
}

template <int INTEG, bool DRAG>
__global__ void __launch_bounds__(256) k_plain_integrate(FleetBuffers fb, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fb.n) return;
  const uint32_t n = fb.n;
  VState s = load_state(fb.state, n, i);
  Wrench4 W = {fb.wrench[0 * n + i], fb.wrench[1 * n + i], fb.wrench[2 * n + i], fb.wrench[3 * n + i]};
  integrate<INTEG, DRAG>(s, body_z(s.q), W, load_body(fb.body, n, i), P);
  store_state(fb.state, n, i, s);
}

// Collision test of every environment against its boxes read from global
// memory; the per-env hit byte goes to `collided_now`.
__global__ void __launch_bounds__(256) k_plain_collide(FleetBuffers fb, StepParams P, uint8_t* collided_now) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fb.n) return;
  const uint32_t n = fb.n;
  V3 p = {fb.state[0 * n + i], fb.state[1 * n + i], fb.state[2 * n + i]};
  bool hit = false;
  for (uint32_t k = 0; k < fb.n_obs; ++k) {
    const float* bx = fb.boxes + (size_t)k * 10 * n + i;
    hit |= sphere_hits_box(p, P.r2, V3{bx[0], bx[n], bx[2 * n]}, V3{bx[3 * n], bx[4 * n], bx[5 * n]},
                           Q4{bx[6 * n], bx[7 * n], bx[8 * n], bx[9 * n]});
  }
  collided_now[i] = hit ? 1 : 0;
}

__global__ void __launch_bounds__(256) k_plain_reset_hits(FleetBuffers fb, StepParams P, const uint8_t* collided_now) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fb.n || collided_now[i] == 0) return;
  const uint32_t n = fb.n;
  const uint32_t epoch = fb.epoch[i] + 1u;
  fb.epoch[i] = epoch;
  fb.resets[i] += 1u;
  fb.collided[i] = 1;
  ResetValues r = draw_reset(P.seed_lo, P.seed_hi, i, epoch);
  float* st = fb.state;
  st[0 * n + i] = r.p[0]; st[1 * n + i] = r.p[1]; st[2 * n + i] = r.p[2];
  st[3 * n + i] = r.v[0]; st[4 * n + i] = r.v[1]; st[5 * n + i] = r.v[2];
  st[6 * n + i] = r.q[0]; st[7 * n + i] = r.q[1]; st[8 * n + i] = r.q[2]; st[9 * n + i] = r.q[3];
  st[10 * n + i] = 0.f; st[11 * n + i] = 0.f; st[12 * n + i] = 0.f;
  const int nrot = rotor_count(fb, i);
  const float hv = hover_per_motor(fb.body[i], nrot);
  for (int k = 0; k < nrot; ++k) fb.motors[k * n + i] = hv;
  if (fb.box_rand) redraw_boxes(fb, i, fb.slot_of ? fb.slot_of[i] : i, epoch, P.seed_lo, P.seed_hi, NoBoxes{});
}

__global__ void __launch_bounds__(256) k_plain_compact(FleetBuffers fb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool pred = i < fb.n && fb.resets[i] > 0u;
  append_compact(pred, i, fb.reset_ids, fb.n_reset);
}

template <int INTEG, bool QUAD_ONLY, bool DRAG, int BOXES>
cudaError_t launch_fused_b(const FleetBuffers& fb, const StepParams& P, int n_steps, int substeps, int B,
                           cudaStream_t st) {
  const auto kernel = k_fused_step<INTEG, QUAD_ONLY, DRAG, BOXES>;
  // raise the dynamic shared-memory cap once per instantiation and device (the attribute is per device)
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemCap);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit, std::memory_order_release);
  }
  if (B == 0) {  // the block size with the most resident warps per SM (ties: the earlier candidate)
    int best = -1;
    for (int b : {64, 128, 96, 32}) {
      const size_t sm = BOXES == kBoxesStaged ? fused_smem_bytes((int)fb.n_obs, b) : 0;
      if (sm > kFusedSmemCap) continue;
      int blocks = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, b, sm);
      if (e != cudaSuccess) return e;
      if (blocks * b > best) { best = blocks * b; B = b; }
    }
    if (best <= 0) return cudaErrorInvalidConfiguration;
  }
  const size_t smem = BOXES == kBoxesStaged ? fused_smem_bytes((int)fb.n_obs, B) : 0;
  const unsigned grid = (fb.n + B - 1) / B;
  kernel<<<grid, B, smem, st>>>(fb, P, n_steps, substeps);
  return cudaGetLastError();
}

template <int INTEG, bool QUAD_ONLY, bool DRAG>
cudaError_t launch_fused_t(const FleetBuffers& fb, const StepParams& P, int n_steps, int substeps, int B,
                           cudaStream_t st) {
  if (fb.n_obs == 0) return launch_fused_b<INTEG, QUAD_ONLY, DRAG, kBoxesNone>(fb, P, n_steps, substeps, B, st);
  // the global pair copy is in slot order: it serves the grouped order only
  if (fb.order && fb.boxes_slot && !fused_boxes_staged_from_env())
    return launch_fused_b<INTEG, QUAD_ONLY, DRAG, kBoxesGlobal>(fb, P, n_steps, substeps, B, st);
  return launch_fused_b<INTEG, QUAD_ONLY, DRAG, kBoxesStaged>(fb, P, n_steps, substeps, B, st);
}

template <int INTEG>
cudaError_t launch_fused_i(const FleetBuffers& fb, const StepParams& P, int n_steps, int substeps, int B,
                           cudaStream_t st) {
  const bool quad_only = fb.n_quad == fb.n;
  const bool drag = P.drag != 0.f;
  if (quad_only)
    return drag ? launch_fused_t<INTEG, true, true>(fb, P, n_steps, substeps, B, st)
                : launch_fused_t<INTEG, true, false>(fb, P, n_steps, substeps, B, st);
  return drag ? launch_fused_t<INTEG, false, true>(fb, P, n_steps, substeps, B, st)
              : launch_fused_t<INTEG, false, false>(fb, P, n_steps, substeps, B, st);
}

}  // namespace

FusedTuning fused_tuning_from_env(int n_obs) {
  FusedTuning t;
  t.sorted = true;
  t.block = 0;
  t.skip = true;
  if (const char* v = std::getenv("AG_FUSED_ORDER")) t.sorted = std::strcmp(v, "identity") != 0;
  if (const char* v = std::getenv("AG_FUSED_SKIP")) t.skip = std::strcmp(v, "0") != 0;
  if (const char* v = std::getenv("AG_FUSED_BLOCK")) {
    int b = std::atoi(v);
    if (b >= 32 && b <= 128 && b % 32 == 0 && fused_smem_bytes(n_obs, b) <= kFusedSmemCap) t.block = b;
  }
  return t;
}

cudaError_t launch_fused_step(const FleetBuffers& fb_in, const StepParams& P, int integrator, int n_steps,
                              int substeps, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(fb_in.n_reset, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess && fb_in.tests_run) e = cudaMemsetAsync(fb_in.tests_run, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const FusedTuning t = fused_tuning_from_env((int)fb_in.n_obs);
  FleetBuffers fb = fb_in;
  if (!t.sorted) fb.order = nullptr;
  StepParams Pl = P;
  if (!t.skip) Pl.exact_tests = 1;
  return integrator == kIntegRK4 ? launch_fused_i<kIntegRK4>(fb, Pl, n_steps, substeps, t.block, st)
                                 : launch_fused_i<kIntegSIE>(fb, Pl, n_steps, substeps, t.block, st);
}

cudaError_t launch_build_order(const FleetBuffers& fb, uint32_t* scratch, cudaStream_t st) {
  (void)scratch;
  k_order_window<<<(fb.n + kOrderWindow - 1) / kOrderWindow, kOrderThreads, 0, st>>>(fb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_permute_boxes(fb, st);
}

size_t order_scratch_words(uint32_t n) {
  (void)n;
  return 1;
}

cudaError_t launch_permute_boxes(const FleetBuffers& fb, cudaStream_t st) {
  if (fb.n_obs == 0 || !fb.order || !fb.boxes_slot) return cudaSuccess;
  k_permute_boxes<<<(fb.n + 255) / 256, 256, 0, st>>>(fb);
  return cudaGetLastError();
}

cudaError_t launch_reset(const FleetBuffers& fb, const uint8_t* mask, uint32_t seed_lo, uint32_t seed_hi,
                         cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(fb.n_reset, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (fb.n + 255) / 256;
  k_reset<<<grid, 256, 0, st>>>(fb, mask, seed_lo, seed_hi);
  return cudaGetLastError();
}

cudaError_t launch_controller(const FleetBuffers& fb, const StepParams& P, cudaStream_t st) {
  k_plain_controller<<<(fb.n + 255) / 256, 256, 0, st>>>(fb, P);
  return cudaGetLastError();
}

cudaError_t launch_plain_step(const FleetBuffers& fb, const StepParams& P, int integrator, int n_steps,
                              int substeps, cudaStream_t st) {
  const unsigned grid = (fb.n + 255) / 256;
  cudaError_t e = cudaMemsetAsync(fb.n_reset, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fb.resets, 0, sizeof(uint32_t) * fb.n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fb.collided, 0, fb.n, st);
  if (e != cudaSuccess) return e;
  uint8_t* hits = fb.hits;
  for (int step = 0; step < n_steps; ++step) {
    for (int ss = 0; ss < substeps; ++ss) {
      k_plain_controller<<<grid, 256, 0, st>>>(fb, P);
      k_plain_allocate<<<grid, 256, 0, st>>>(fb, P);
      const bool drag = P.drag != 0.f;
      if (integrator == kIntegRK4) {
        if (drag) k_plain_integrate<kIntegRK4, true><<<grid, 256, 0, st>>>(fb, P);
        else k_plain_integrate<kIntegRK4, false><<<grid, 256, 0, st>>>(fb, P);
      } else {
        if (drag) k_plain_integrate<kIntegSIE, true><<<grid, 256, 0, st>>>(fb, P);
        else k_plain_integrate<kIntegSIE, false><<<grid, 256, 0, st>>>(fb, P);
      }
    }
    if (fb.n_obs > 0) {
      k_plain_collide<<<grid, 256, 0, st>>>(fb, P, hits);
      k_plain_reset_hits<<<grid, 256, 0, st>>>(fb, P, hits);
    }
  }
  k_plain_compact<<<grid, 256, 0, st>>>(fb);
  return cudaGetLastError();
}

}  // namespace agk
