// fleet_sim.cuh — the per-vehicle loop shared by the fused kernels.
//
// Loading one environment into registers, running its steps (controller,
// allocation, integrator, collision test, in-register Philox reset) and
// storing it back; plus the warp-level compaction of reset ids. Used by the
// single-fleet fused kernel and by the multi-request serving kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fleet_device.cuh"
#include "fleet_internal.h"
#include "reset_sampler.cuh"

namespace agk {

__device__ __forceinline__ int rotor_count(const FleetBuffers& fb, uint32_t env) {
  if (env < fb.n_quad) return 4;
  if (env < fb.n_quad + fb.n_hexa) return 6;
  return 8;
}

__device__ __forceinline__ VState load_state(const float* st, uint32_t n, uint32_t i) {
  VState s;
  s.p = {st[0 * n + i], st[1 * n + i], st[2 * n + i]};
  s.v = {st[3 * n + i], st[4 * n + i], st[5 * n + i]};
  s.q = {st[6 * n + i], st[7 * n + i], st[8 * n + i], st[9 * n + i]};
  s.w = {st[10 * n + i], st[11 * n + i], st[12 * n + i]};
  return s;
}

__device__ __forceinline__ void store_state(float* st, uint32_t n, uint32_t i, const VState& s) {
  st[0 * n + i] = s.p.x; st[1 * n + i] = s.p.y; st[2 * n + i] = s.p.z;
  st[3 * n + i] = s.v.x; st[4 * n + i] = s.v.y; st[5 * n + i] = s.v.z;
  st[6 * n + i] = s.q.w; st[7 * n + i] = s.q.x; st[8 * n + i] = s.q.y; st[9 * n + i] = s.q.z;
  st[10 * n + i] = s.w.x; st[11 * n + i] = s.w.y; st[12 * n + i] = s.w.z;
}

__device__ __forceinline__ Body load_body(const float* bd, uint32_t n, uint32_t i) {
  return make_body(bd[0 * n + i], bd[1 * n + i], bd[2 * n + i], bd[3 * n + i]);
}

__device__ __forceinline__ Command load_command(const FleetBuffers& fb, uint32_t i) {
  const uint32_t n = fb.n;
  return prepare_command(fb.modes[i], fb.targets[0 * n + i], fb.targets[1 * n + i], fb.targets[2 * n + i],
                         fb.targets[3 * n + i]);
}

// Overwrites one environment with its reset draw for `epoch`.
template <int NROT>
__device__ __forceinline__ void reset_in_registers(VState& s, float (&u)[NROT], float m, uint32_t env,
                                                   uint32_t epoch, uint32_t seed_lo, uint32_t seed_hi) {
  ResetValues r = draw_reset(seed_lo, seed_hi, env, epoch);
  s.p = {r.p[0], r.p[1], r.p[2]};
  s.v = {r.v[0], r.v[1], r.v[2]};
  s.q = {r.q[0], r.q[1], r.q[2], r.q[3]};
  s.w = {0.f, 0.f, 0.f};
  float hv = hover_per_motor(m, NROT);
#pragma unroll
  for (int k = 0; k < NROT; ++k) u[k] = hv;
}

// Appends the envs whose predicate is set to the compact list: one ballot and
// one atomicAdd per warp, ranks from __popc of the lower lanes. Every lane of
// the warp must call it.
__device__ __forceinline__ void append_compact(bool pred, uint32_t env, uint32_t* ids, uint32_t* count) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
  if (mask == 0u) return;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if ((int)lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (pred) ids[base + __popc(mask & ((1u << lane) - 1u))] = env;
}

// Box sources of the per-vehicle loop; any_hit_min(p, r2, n_obs, m) runs the
// sphere-vs-box test against all boxes of the environment and leaves the
// smallest squared distance to a box in m, staged() is the copy a re-draw
// updates and reload() re-reads what a re-draw changed.
//
// Boxes are handled in pairs (field f of boxes 2j and 2j+1 side by side), so
// one 8-byte load fetches a field of two boxes and the test runs on both at
// once with Blackwell's packed FP32x2 arithmetic. An odd box count is padded
// with a box at 1e30 that cannot be touched.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Field f of the padding box that completes an odd box count: centre at
// 1e30, zero extents, identity orientation (no sphere can touch it).
__device__ __forceinline__ float box_pad_field(int f) { return f < 3 ? 1e30f : (f == 6 ? 1.f : 0.f); }

// Staged form of box field f in the pair copies (the slot-ordered copy and
// each thread's staged copy): the centre, the half-extents and the
// orientation's scalar part are held negated (-c, -h, -w) and its vector
// part doubled (2u). Both are exact, and pair_hits then needs no negation
// and no factor 2.
__device__ __forceinline__ float staged_field(int f, float v) { return f >= 7 ? 2.f * v : -v; }

// Sphere (squared radius r2, centre p) against two boxes at once; the ten
// float2 hold (box a, box b) of the staged fields (see staged_field): -c,
// -h, -w and 2u. With v = p - c and t = 2 u x v, the box-frame point
// d = R_b^T v = v - w t + u x t is computed as (v - w t) + 1/2 ((2u) x t);
// negation, doubling and halving are exact, so d rounds as the plain form
// would.
// Returns the squared distances from p to the two boxes.
__device__ __forceinline__ float2 pair_dist2(float2 px, float2 py, float2 pz, float2 ncx, float2 ncy, float2 ncz,
                                             float2 nhx, float2 nhy, float2 nhz, float2 nqw, float2 ux2, float2 uy2,
                                             float2 uz2) {
  const float2 vx = add2(px, ncx), vy = add2(py, ncy), vz = add2(pz, ncz);
  const float2 tx = fma2(uy2, vz, neg2(mul2(uz2, vy)));
  const float2 ty = fma2(uz2, vx, neg2(mul2(ux2, vz)));
  const float2 tz = fma2(ux2, vy, neg2(mul2(uy2, vx)));
  const float2 half = dup2(0.5f);
  const float2 dx = fma2(half, fma2(uy2, tz, neg2(mul2(uz2, ty))), fma2(nqw, tx, vx));
  const float2 dy = fma2(half, fma2(uz2, tx, neg2(mul2(ux2, tz))), fma2(nqw, ty, vy));
  const float2 dz = fma2(half, fma2(ux2, ty, neg2(mul2(uy2, tx))), fma2(nqw, tz, vz));
  // excess over the half-extents, clamped at 0
  const float2 ex = add2(make_float2(fabsf(dx.x), fabsf(dx.y)), nhx);
  const float2 ey = add2(make_float2(fabsf(dy.x), fabsf(dy.y)), nhy);
  const float2 ez = add2(make_float2(fabsf(dz.x), fabsf(dz.y)), nhz);
  const float2 mx = make_float2(fmaxf(ex.x, 0.f), fmaxf(ex.y, 0.f));
  const float2 my = make_float2(fmaxf(ey.x, 0.f), fmaxf(ey.y, 0.f));
  const float2 mz = make_float2(fmaxf(ez.x, 0.f), fmaxf(ez.y, 0.f));
  return fma2(mz, mz, fma2(my, my, mul2(mx, mx)));
}

// Sphere (squared radius r2, centre p) against two boxes at once: touching
// counts.
__device__ __forceinline__ bool pair_hits(float2 px, float2 py, float2 pz, float r2, float2 ncx, float2 ncy,
                                          float2 ncz, float2 nhx, float2 nhy, float2 nhz, float2 nqw, float2 ux2,
                                          float2 uy2, float2 uz2) {
  const float2 e2 = pair_dist2(px, py, pz, ncx, ncy, ncz, nhx, nhy, nhz, nqw, ux2, uy2, uz2);
  return !(r2 < e2.x) | !(r2 < e2.y);
}

// The pair test that also lowers m to the smaller squared distance.
__device__ __forceinline__ bool pair_hits_min(float2 px, float2 py, float2 pz, float r2, float2 ncx, float2 ncy,
                                              float2 ncz, float2 nhx, float2 nhy, float2 nhz, float2 nqw, float2 ux2,
                                              float2 uy2, float2 uz2, float& m) {
  const float2 e2 = pair_dist2(px, py, pz, ncx, ncy, ncz, nhx, nhy, nhz, nqw, ux2, uy2, uz2);
  m = fminf(m, fminf(e2.x, e2.y));
  return !(r2 < e2.x) | !(r2 < e2.y);
}

// RegSmemBoxPairs: the first pair (boxes 0 and 1) in registers, the others
// in shared memory as float4 [pair - 1][field pair][thread], each float4 two
// consecutive fields of both boxes, (a_f, b_f, a_f+1, b_f+1): a pair is five
// 16-byte loads, and a warp's load of one float4 row is 512 consecutive bytes
// (no bank conflicts). Holding one pair in registers shrinks each thread's
// shared-memory footprint by a tenth of the 16-box case, which lets one more
// block reside per SM.
struct RegSmemBoxPairs {
  float2 r[10];  // pair 0, fields 0..9
  float4* sm;    // this thread's column of pairs 1..: element ((j - 1) * 5 + f / 2) * B
  int B;
  // Any box within r of p; m receives the smallest squared distance to a box.
  __device__ __forceinline__ bool any_hit_min(V3 p, float r2, int n_obs, float& m) const {
    const float2 px = dup2(p.x), py = dup2(p.y), pz = dup2(p.z);
    m = __int_as_float(0x7f800000);
    bool hit = pair_hits_min(px, py, pz, r2, r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9], m);
    const int pairs = (n_obs + 1) >> 1;
#pragma unroll 2
    for (int j = 1; j < pairs; ++j) {
      const float4* f = sm + (size_t)(j - 1) * 5 * B;
      const float4 f01 = f[0], f23 = f[B], f45 = f[2 * B], f67 = f[3 * B], f89 = f[4 * B];
      hit |= pair_hits_min(px, py, pz, r2, make_float2(f01.x, f01.y), make_float2(f01.z, f01.w),
                           make_float2(f23.x, f23.y), make_float2(f23.z, f23.w), make_float2(f45.x, f45.y),
                           make_float2(f45.z, f45.w), make_float2(f67.x, f67.y), make_float2(f67.z, f67.w),
                           make_float2(f89.x, f89.y), make_float2(f89.z, f89.w), m);
    }
    return hit;
  }
  // The shared-memory part, as the target of a re-draw (boxes 2..).
  struct Staged {
    float4* sm;
    int B;
    __device__ __forceinline__ void set(int k, int f, float v) const {
      if (k < 2) return;
      float4& e = sm[(size_t)(((k >> 1) - 1) * 5 + (f >> 1)) * B];
      const int c = (f & 1) * 2 + (k & 1);  // a_f, b_f, a_f+1, b_f+1
      if (c == 0) e.x = v; else if (c == 1) e.y = v; else if (c == 2) e.z = v; else e.w = v;
    }
  };
  __device__ __forceinline__ Staged staged() const { return {sm, B}; }
  // pair 0 from the env-ordered boxes (after a re-draw)
  __device__ __forceinline__ void reload(const FleetBuffers& fb, uint32_t env) {
    const uint32_t n = fb.n;
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      r[f].x = staged_field(f, fb.boxes[(size_t)f * n + env]);
      r[f].y = staged_field(f, fb.n_obs > 1 ? fb.boxes[(size_t)(10 + f) * n + env] : box_pad_field(f));
    }
  }
};

// No staged copy (kernels that only update the global boxes).
struct NoBoxes {
  __device__ __forceinline__ void set(int, int, float) const {}
};

// No boxes at all (a fleet without obstacles): nothing to test or re-load.
struct NoBoxSource {
  __device__ __forceinline__ bool any_hit_min(V3, float, int, float& m) const {
    m = __int_as_float(0x7f800000);
    return false;
  }
  __device__ __forceinline__ NoBoxes staged() const { return {}; }
  __device__ __forceinline__ void reload(const FleetBuffers&, uint32_t) {}
};

// GlobalBoxPairs: the slot-ordered pair copy in global memory, element
// (j * 10 + f) * n + idx, read through the read-only cache.
struct GlobalBoxPairs {
  const float2* __restrict__ rows;
  uint32_t n, idx;
  // a re-draw refreshes the global copy itself; nothing is cached here
  __device__ __forceinline__ void set(int, int, float) const {}
  __device__ __forceinline__ NoBoxes staged() const { return {}; }
  __device__ __forceinline__ void reload(const FleetBuffers&, uint32_t) {}
  __device__ __forceinline__ float2 at(int r) const { return __ldg(rows + (size_t)r * n + idx); }
  __device__ __forceinline__ bool any_hit_min(V3 p, float r2, int n_obs, float& m) const {
    const float2 px = dup2(p.x), py = dup2(p.y), pz = dup2(p.z);
    bool hit = false;
    m = __int_as_float(0x7f800000);
    const int pairs = (n_obs + 1) >> 1;
#pragma unroll 2
    for (int j = 0; j < pairs; ++j) {
      const int r = j * 10;
      hit |= pair_hits_min(px, py, pz, r2, at(r), at(r + 1), at(r + 2), at(r + 3), at(r + 4), at(r + 5), at(r + 6),
                           at(r + 7), at(r + 8), at(r + 9), m);
    }
    return hit;
  }
};

// The per-vehicle body of the fused kernels, specialised on the rotor count:
// n_steps steps of `substeps` substeps, then the sphere-vs-box test against
// n_obs boxes and, on a hit, the Philox reset keyed (seed_lo, seed_hi).
// New poses for every box of environment env (slot = its thread slot):
// written to the env-ordered boxes, to the slot-ordered pair copy and to the
// caller's box source (the thread's staged copy).
template <class Boxes>
__device__ __noinline__ void redraw_boxes(const FleetBuffers& fb, uint32_t env, uint32_t slot, uint32_t epoch,
                                          uint32_t seed_lo, uint32_t seed_hi, const Boxes& boxes) {
  const uint32_t n = fb.n;
  for (int k = 0; k < (int)fb.n_obs; ++k) {
    float c[3], q[4];
    draw_box_pose(seed_lo, seed_hi, env, epoch, (uint32_t)k, fb.box_rand[k], c, q);
    const float v[7] = {c[0], c[1], c[2], q[0], q[1], q[2], q[3]};
    const int field[7] = {0, 1, 2, 6, 7, 8, 9};
    for (int m = 0; m < 7; ++m) {
      const int f = field[m];
      fb.boxes[((size_t)k * 10 + f) * n + env] = v[m];
      const float sv = staged_field(f, v[m]);
      if (fb.boxes_slot) {
        float2& e = fb.boxes_slot[(size_t)((k >> 1) * 10 + f) * n + slot];
        if (k & 1) e.y = sv; else e.x = sv;
      }
      boxes.set(k, f, sv);
    }
  }
}

// Resets environment env in device memory (the ag_reset draw): epoch + 1,
// Philox state draw, every motor at hover, zero for the unused ones, and new
// box poses when re-placement is on.
__device__ __forceinline__ void reset_env(const FleetBuffers& fb, uint32_t env, uint32_t seed_lo, uint32_t seed_hi) {
  const uint32_t n = fb.n;
  const uint32_t epoch = fb.epoch[env] + 1u;
  fb.epoch[env] = epoch;
  ResetValues r = draw_reset(seed_lo, seed_hi, env, epoch);
  float* st = fb.state;
  st[0 * n + env] = r.p[0]; st[1 * n + env] = r.p[1]; st[2 * n + env] = r.p[2];
  st[3 * n + env] = r.v[0]; st[4 * n + env] = r.v[1]; st[5 * n + env] = r.v[2];
  st[6 * n + env] = r.q[0]; st[7 * n + env] = r.q[1]; st[8 * n + env] = r.q[2]; st[9 * n + env] = r.q[3];
  st[10 * n + env] = 0.f; st[11 * n + env] = 0.f; st[12 * n + env] = 0.f;
  const int nrot = rotor_count(fb, env);
  const float hv = hover_per_motor(fb.body[env], nrot);
  for (int k = 0; k < 8; ++k) fb.motors[k * n + env] = k < nrot ? hv : 0.f;
  if (fb.box_rand) redraw_boxes(fb, env, fb.slot_of ? fb.slot_of[env] : env, epoch, seed_lo, seed_hi, NoBoxes{});
}

// How far a vehicle may move from p, where the exact test found min_e2 as
// its smallest squared distance to a box, before the sphere of radius r could
// touch one; returned squared, or -1 when it must be tested again at once.
// The distance to a box is 1-Lipschitz in the position, so as long as
// |p' - p| < sqrt(min_e2) - r - slack no box is within r of p'. The slack
// (1 mm plus 1e-5 of the magnitudes involved) is far above the float32
// rounding of the test, so a skipped test is one the exact float32 test
// would also have found clear: every collision decision is the exact test's.
__device__ __forceinline__ float clearance_threshold2(V3 p, float min_e2, float r) {
  const float c = sqrtf(min_e2) - r;
  const float slack = 1e-3f + 1e-5f * (fabsf(c) + fabsf(p.x) + fabsf(p.y) + fabsf(p.z));
  const float t = c - slack;
  return t > 0.f ? t * t : -1.f;
}

// simulate() with the command given (cm_in) instead of read from fb; returns
// the final state, which it also stores. MODE >= 0: every calling thread's
// command mode is MODE; the mode is then a constant of the compiled loop,
// and the controller's branches on it fold away.
template <int NROT, int INTEG, bool DRAG, class Boxes, int MODE = -1>
__device__ __forceinline__ VState simulate_cmd(const FleetBuffers& fb, const StepParams& P, uint32_t env,
                                               uint32_t slot, const Command& cm_in, int n_steps, int substeps, int n_obs,
                                               Boxes& boxes, uint32_t seed_lo, uint32_t seed_hi, uint32_t& resets,
                                               bool& any_hit, uint32_t& tests) {
  Command cm = cm_in;
  if (MODE >= 0) cm.mode = MODE;
  const uint32_t n = fb.n;
  VState s = load_state(fb.state, n, env);
  normalize(s.q);
  float u[NROT];
#pragma unroll
  for (int k = 0; k < NROT; ++k) u[k] = fb.motors[k * n + env];
  const Body b = load_body(fb.body, n, env);
  uint32_t epoch = fb.epoch[env];
  // Collision tests that cannot hit are skipped (see clearance_threshold2):
  // p_test is the position of the last exact test, thr2 the squared distance
  // the vehicle may move from there before it could touch a box (-1: test
  // at the next step).
  V3 p_test = {0.f, 0.f, 0.f};
  float thr2 = -1.f;
  const float r = sqrtf(P.r2);
  for (int step = 0; step < n_steps; ++step) {
    for (int ss = 0; ss < substeps; ++ss) {
      V3 b3;
      Wrench4 W = allocate<NROT>(controller(s, cm, b, P, b3), u, P);
      integrate<INTEG, DRAG>(s, b3, W, b, P);
    }
    if (n_obs > 0) {
      const V3 dp = s.p - p_test;
      if (!(dot(dp, dp) < thr2)) {
        float min_e2;
        const bool hit = boxes.any_hit_min(s.p, P.r2, n_obs, min_e2);
        tests += 1;
        p_test = s.p;
        thr2 = P.exact_tests ? -1.f : clearance_threshold2(s.p, min_e2, r);
        if (hit) {
          any_hit = true;
          resets += 1;
          epoch += 1;
          reset_in_registers<NROT>(s, u, b.m, env, epoch, seed_lo, seed_hi);
          thr2 = -1.f;
          if (fb.box_rand) {
            redraw_boxes(fb, env, slot, epoch, seed_lo, seed_hi, boxes.staged());
            boxes.reload(fb, env);
          }
        }
      }
    }
  }
  store_state(fb.state, n, env, s);
#pragma unroll
  for (int k = 0; k < NROT; ++k) fb.motors[k * n + env] = u[k];
  fb.epoch[env] = epoch;
  return s;
}

// With BY_MODE and the grouped thread order (fb.order: warps of one rotor
// count and command mode), a group of threads that run together and share
// one command mode (position, body velocity, attitude + thrust) runs the
// steps compiled for that mode, in which the controller's branches on the
// mode are folded away; other threads run the branching form. Every fused
// multiply-add of the step is explicit (fmaf) and the files that include
// this header are compiled without contraction, so both forms round
// identically and the choice changes no result.
template <int NROT, int INTEG, bool DRAG, bool BY_MODE = false, class Boxes>
__device__ __forceinline__ void simulate(const FleetBuffers& fb, const StepParams& P, uint32_t env, uint32_t slot,
                                         int n_steps, int substeps, int n_obs, Boxes& boxes, uint32_t seed_lo,
                                         uint32_t seed_hi, uint32_t& resets, bool& any_hit, uint32_t& tests) {
  const Command cm = load_command(fb, env);
  bool uniform = false;
  if (BY_MODE && fb.order) {
    const unsigned group = __activemask();
    uniform = __match_any_sync(group, cm.mode) == group;
  }
  if (uniform) {
    if (cm.mode == kModePosition) {
      simulate_cmd<NROT, INTEG, DRAG, Boxes, kModePosition>(fb, P, env, slot, cm, n_steps, substeps, n_obs, boxes,
                                                           seed_lo, seed_hi, resets, any_hit, tests);
      return;
    }
    if (cm.mode == kModeBodyVel) {
      simulate_cmd<NROT, INTEG, DRAG, Boxes, kModeBodyVel>(fb, P, env, slot, cm, n_steps, substeps, n_obs, boxes,
                                                          seed_lo, seed_hi, resets, any_hit, tests);
      return;
    }
    if (cm.mode == kModeAttThrust) {
      simulate_cmd<NROT, INTEG, DRAG, Boxes, kModeAttThrust>(fb, P, env, slot, cm, n_steps, substeps, n_obs, boxes,
                                                            seed_lo, seed_hi, resets, any_hit, tests);
      return;
    }
  }
  simulate_cmd<NROT, INTEG, DRAG>(fb, P, env, slot, cm, n_steps, substeps, n_obs, boxes, seed_lo, seed_hi, resets,
                                  any_hit, tests);
}

}  // namespace agk
