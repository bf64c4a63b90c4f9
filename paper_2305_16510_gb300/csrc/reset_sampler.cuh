// reset_sampler.cuh — device Philox4x32-10 and the strict-binary32 reset draw.
//
// Resetting an environment (Kulkarni et al., arXiv 2305.16510, Sec. V: the
// asset manager samples a new pose when an environment resets) draws from the
// counter-based generator Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011),
// implemented here from that definition. Each draw is a pure function of
// (seed, env, epoch): counter (env, epoch, slot, 0), key (seed lo, seed hi).
// The transform from words to values uses only round-to-nearest binary32
// intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn) and integer ops, so
// the compiler cannot contract or reassociate it and every build on every GPU
// produces the same bits.
//
// Word use per slot (w0..w3):
//   slot 0: position x, y, z ~ U[-2, 2);  axis z ~ U(-1, 1]
//   slot 1: axis azimuth, rotation angle, Box-Muller pair 1 (log word, turn word)
//   slot 2: Box-Muller pair 2 (log word, turn word)
// attitude = rotation by U[0, pi/6) about the axis; velocity ~ N(0, 0.5^2):
// v_x, v_y from pair 1 (cos, sin), v_z from pair 2 (cos).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace agk {

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x), lo0 = 0xD2511F53u * ctr.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z), lo1 = 0xCD9E8D57u * ctr.z;
    ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return ctr;
}

// top 24 bits as a binary32 in [0, 1): exact
__device__ __forceinline__ float unit24(uint32_t w) { return __fmul_rn(__uint2float_rn(w >> 8), 0x1.0p-24f); }

// sin, cos of |h| <= pi/2: Taylor polynomials to degree 13 / 14, Horner in h^2
__device__ __forceinline__ void sincos_taylor(float h, float* sn, float* cs) {
  float h2 = __fmul_rn(h, h);
  float s = -0x1.612462p-33f;
  s = __fadd_rn(__fmul_rn(s, h2), 0x1.ae6456p-26f);
  s = __fadd_rn(__fmul_rn(s, h2), -0x1.71de3ap-19f);
  s = __fadd_rn(__fmul_rn(s, h2), 0x1.a01a02p-13f);
  s = __fadd_rn(__fmul_rn(s, h2), -0x1.111112p-7f);
  s = __fadd_rn(__fmul_rn(s, h2), 0x1.555556p-3f);
  float c = 0x1.93974ap-37f;
  c = __fadd_rn(__fmul_rn(c, h2), -0x1.1eed8ep-29f);
  c = __fadd_rn(__fmul_rn(c, h2), 0x1.27e4fcp-22f);
  c = __fadd_rn(__fmul_rn(c, h2), -0x1.a01a02p-16f);
  c = __fadd_rn(__fmul_rn(c, h2), 0x1.6c16c2p-10f);
  c = __fadd_rn(__fmul_rn(c, h2), -0x1.555556p-5f);
  c = __fadd_rn(__fmul_rn(c, h2), 0x1.0p-1f);
  *sn = __fsub_rn(h, __fmul_rn(__fmul_rn(h, h2), s));
  *cs = __fsub_rn(1.0f, __fmul_rn(h2, c));
}

// cos and sin of 2 pi (w >> 8) / 2^24: quadrant from the top two bits
__device__ __forceinline__ void sincos_of_turn(uint32_t w, float* cs, float* sn) {
  uint32_t k = w >> 8;
  float h = __fmul_rn(__uint2float_rn(k & 0x3FFFFFu), 0x1.921fb6p-22f);
  float s, c;
  sincos_taylor(h, &s, &c);
  switch (k >> 22) {
    case 0: *cs = c; *sn = s; break;
    case 1: *cs = -s; *sn = c; break;
    case 2: *cs = -c; *sn = -s; break;
    default: *cs = s; *sn = -c; break;
  }
}

// ln((k + 1) 2^-24), k = w >> 8: exponent split, atanh series to s^11
__device__ __forceinline__ float log_unit24(uint32_t w) {
  uint32_t m = (w >> 8) + 1u;
  int e = 31 - __clz(m);
  float f = __fmul_rn(__uint2float_rn(m), __int_as_float((127 - e) << 23));
  if (f > 0x1.6a09e6p+0f) {
    f = __fmul_rn(f, 0.5f);
    e += 1;
  }
  float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  float s2 = __fmul_rn(s, s);
  float p = 0x1.745d18p-4f;
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.c71c72p-4f);
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.24924ap-3f);
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.99999ap-3f);
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.555556p-2f);
  p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
  float lnf = __fmul_rn(__fmul_rn(2.0f, s), p);
  return __fadd_rn(__fmul_rn(__int2float_rn(e - 24), 0x1.62e430p-1f), lnf);
}

struct ResetValues { float p[3], v[3], q[4]; };

__device__ __forceinline__ ResetValues draw_reset(uint32_t seed_lo, uint32_t seed_hi, uint32_t env, uint32_t epoch) {
  uint4 w0 = philox4x32_10(make_uint4(env, epoch, 0u, 0u), seed_lo, seed_hi);
  uint4 w1 = philox4x32_10(make_uint4(env, epoch, 1u, 0u), seed_lo, seed_hi);
  uint4 w2 = philox4x32_10(make_uint4(env, epoch, 2u, 0u), seed_lo, seed_hi);
  ResetValues r;
  r.p[0] = __fadd_rn(-2.0f, __fmul_rn(4.0f, unit24(w0.x)));
  r.p[1] = __fadd_rn(-2.0f, __fmul_rn(4.0f, unit24(w0.y)));
  r.p[2] = __fadd_rn(-2.0f, __fmul_rn(4.0f, unit24(w0.z)));
  float az = __fsub_rn(1.0f, __fmul_rn(2.0f, unit24(w0.w)));
  float om = __fsub_rn(1.0f, __fmul_rn(az, az));
  float rho = om > 0.0f ? __fsqrt_rn(om) : 0.0f;
  float ca, sa;
  sincos_of_turn(w1.x, &ca, &sa);
  float half = __fmul_rn(unit24(w1.y), 0x1.0c1524p-2f);
  float sh, ch;
  sincos_taylor(half, &sh, &ch);
  r.q[0] = ch;
  r.q[1] = __fmul_rn(sh, __fmul_rn(rho, ca));
  r.q[2] = __fmul_rn(sh, __fmul_rn(rho, sa));
  r.q[3] = __fmul_rn(sh, az);
  float r1 = __fsqrt_rn(__fmul_rn(-2.0f, log_unit24(w1.z)));
  float c1, s1;
  sincos_of_turn(w1.w, &c1, &s1);
  float r2 = __fsqrt_rn(__fmul_rn(-2.0f, log_unit24(w2.x)));
  float c2, s2;
  sincos_of_turn(w2.y, &c2, &s2);
  r.v[0] = __fmul_rn(0.5f, __fmul_rn(r1, c1));
  r.v[1] = __fmul_rn(0.5f, __fmul_rn(r1, s1));
  r.v[2] = __fmul_rn(0.5f, __fmul_rn(r2, c2));
  return r;
}

// Re-draw spec of one obstacle (the layout of ag_box_randomization) with the
// environment bounds appended.
struct BoxRandDev {
  float pos_min[3], pos_max[3];      // fractions of the environment bounds
  float euler_min[3], euler_max[3];  // roll, pitch, yaw [rad]
  uint32_t lock;                     // bit d: dimension d (x, y, z, roll, pitch, yaw) held at fixed[d]
  float fixed[6];
  float env_min[3], env_max[3];
};

// New pose of box k of environment env at epoch (Sec. V: obstacles are
// re-placed when their environment resets). Counter (env, epoch, k, 1) gives
// the x, y, z fractions and the roll; (env, epoch, k, 2) the pitch and yaw.
// q = q_z(yaw) (x) q_y(pitch) (x) q_x(roll) from half-angle sines and cosines.
__device__ __forceinline__ void draw_box_pose(uint32_t seed_lo, uint32_t seed_hi, uint32_t env, uint32_t epoch,
                                              uint32_t k, const BoxRandDev& r, float c[3], float q[4]) {
  const uint4 w1 = philox4x32_10(make_uint4(env, epoch, k, 1u), seed_lo, seed_hi);
  const uint4 w2 = philox4x32_10(make_uint4(env, epoch, k, 2u), seed_lo, seed_hi);
  const uint32_t wp[3] = {w1.x, w1.y, w1.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (r.lock & (1u << d)) {
      c[d] = r.fixed[d];
    } else {
      const float f = __fadd_rn(r.pos_min[d], __fmul_rn(__fsub_rn(r.pos_max[d], r.pos_min[d]), unit24(wp[d])));
      c[d] = __fadd_rn(r.env_min[d], __fmul_rn(__fsub_rn(r.env_max[d], r.env_min[d]), f));
    }
  }
  const uint32_t wa[3] = {w1.w, w2.x, w2.y};
  float sn[3], cs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float ang = (r.lock & (1u << (3 + a)))
                          ? r.fixed[3 + a]
                          : __fadd_rn(r.euler_min[a], __fmul_rn(__fsub_rn(r.euler_max[a], r.euler_min[a]), unit24(wa[a])));
    sincos_taylor(__fmul_rn(0.5f, ang), &sn[a], &cs[a]);
  }
  const float cr = cs[0], sr = sn[0], cp = cs[1], sp = sn[1], cy = cs[2], sy = sn[2];
  const float cycp = __fmul_rn(cy, cp), sysp = __fmul_rn(sy, sp), cysp = __fmul_rn(cy, sp), sycp = __fmul_rn(sy, cp);
  q[0] = __fadd_rn(__fmul_rn(cycp, cr), __fmul_rn(sysp, sr));
  q[1] = __fsub_rn(__fmul_rn(cycp, sr), __fmul_rn(sysp, cr));
  q[2] = __fadd_rn(__fmul_rn(cysp, cr), __fmul_rn(sycp, sr));
  q[3] = __fsub_rn(__fmul_rn(sycp, cr), __fmul_rn(cysp, sr));
}

__device__ __forceinline__ float hover_per_motor(float m, int n_rot) {
  return __fdiv_rn(__fmul_rn(m, 9.81f), __int2float_rn(n_rot));
}

}  // namespace agk
