// philox_sampler.hpp — counter-based reset sampler of the oracle.
//
// TEST INFRASTRUCTURE ONLY (see aerial_oracle.hpp).
//
// Resetting an environment draws a new initial state (Sec. V: the asset
// manager samples positions and orientations when environments reset). The
// draws come from the counter-based generator Philox4x32-10 of Salmon,
// Moraes, Dror & Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3"
// (SC 2011), written here from that paper's definition. The transform from
// random words to state values is defined in strict IEEE-754 binary32 with
// round-to-nearest-even on every operation (this file must be compiled with
// -ffp-contract=off so no multiply-add is fused), using only +, -, *, /,
// sqrt and integer operations. It is therefore reproducible bit for bit by
// any independent implementation that follows the same operation order.
//
// Draw layout: counter = (env_id, epoch, slot, 0), key = (seed mod 2^32,
// seed div 2^32); each slot yields four 32-bit words w0..w3:
//   slot 0: w0, w1, w2 -> position x, y, z ~ U[-2, 2);  w3 -> axis z
//   slot 1: w0 -> axis azimuth,  w1 -> rotation angle,
//           w2, w3 -> first Box-Muller pair (radius word, turn word)
//   slot 2: w0, w1 -> second Box-Muller pair;  w2, w3 unused
// Values: attitude = rotation by an angle U[0, pi/6) about an axis uniform
// on the unit sphere; velocity ~ N(0, 0.5^2) per component (v_x, v_y from
// the first pair's cosine and sine, v_z from the second pair's cosine);
// body rate 0; every motor at hover thrust m * 9.81 / n_rot.
#pragma once

#include <cstdint>
#include <cstring>

namespace orc {

// ------------------------------------------------------- Philox4x32-10 ----
// One round maps (X0, X1, X2, X3) with key (K0, K1) to
//   (hi(M1*X2) ^ X1 ^ K0, lo(M1*X2), hi(M0*X0) ^ X3 ^ K1, lo(M0*X0)),
// and the key is bumped by the Weyl constants between rounds. Ten rounds.
inline void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// ----------------------------------------------- strict FP32 transforms ----
// Uniform on [0, 1) from the top 24 bits: exact (integer < 2^24 times 2^-24).
inline float u01_f32(uint32_t w) { return (float)(w >> 8) * 0x1.0p-24f; }

// sin and cos of h for |h| <= pi/2 from their Taylor series (sin to h^13,
// cos to h^14), evaluated by Horner's rule in h^2.
inline void sincos_poly_f32(float h, float* s_out, float* c_out) {
  float h2 = h * h;
  float s = -0x1.612462p-33f;  // -1/13!
  s = s * h2 + 0x1.ae6456p-26f;   //  1/11!
  s = s * h2 + -0x1.71de3ap-19f;  // -1/9!
  s = s * h2 + 0x1.a01a02p-13f;   //  1/7!
  s = s * h2 + -0x1.111112p-7f;   // -1/5!
  s = s * h2 + 0x1.555556p-3f;    //  1/3!
  float c = 0x1.93974ap-37f;  //  1/14!
  c = c * h2 + -0x1.1eed8ep-29f;  // -1/12!
  c = c * h2 + 0x1.27e4fcp-22f;   //  1/10!
  c = c * h2 + -0x1.a01a02p-16f;  // -1/8!
  c = c * h2 + 0x1.6c16c2p-10f;   //  1/6!
  c = c * h2 + -0x1.555556p-5f;   // -1/4!
  c = c * h2 + 0x1.0p-1f;        //  1/2!
  // s = 1/3! - h^2/5! + h^4/7! - ...,  so sin h = h - h^3 s;
  // c = 1/2! - h^2/4! + h^4/6! - ...,  so cos h = 1 - h^2 c.
  *s_out = h - (h * h2) * s;
  *c_out = 1.0f - h2 * c;
}

// (cos, sin) of the angle 2*pi*k/2^24 with k = w >> 8: the top two bits of k
// pick the quadrant exactly, the low 22 bits give h in [0, pi/2).
inline void sincos_turn_f32(uint32_t w, float* c_out, float* s_out) {
  uint32_t k = w >> 8;
  uint32_t quadrant = k >> 22;
  uint32_t r = k & 0x3FFFFFu;
  float h = (float)r * 0x1.921fb6p-22f;  // (pi/2) * 2^-22 in binary32
  float s, c;
  sincos_poly_f32(h, &s, &c);
  switch (quadrant) {
    case 0: *c_out = c;  *s_out = s;  break;
    case 1: *c_out = -s; *s_out = c;  break;
    case 2: *c_out = -c; *s_out = -s; break;
    default: *c_out = s; *s_out = -c; break;
  }
}

// ln(u) for u = (k + 1) * 2^-24 in (0, 1], k = w >> 8. With m = k + 1 =
// f * 2^e, f in (sqrt(1/2), sqrt(2)], ln f = 2 atanh(s), s = (f-1)/(f+1),
// from the atanh series to s^11; ln u = (e - 24) ln 2 + ln f.
inline float log_u01_f32(uint32_t w) {
  uint32_t m = (w >> 8) + 1u;  // 1 .. 2^24
  int e = 31;
  while (((m >> e) & 1u) == 0u) --e;  // e = floor(log2 m)
  uint32_t bits = (uint32_t)(127 - e) << 23;
  float two_pow_minus_e;
  std::memcpy(&two_pow_minus_e, &bits, sizeof(float));
  float f = (float)m * two_pow_minus_e;  // exact, in [1, 2)
  if (f > 0x1.6a09e6p+0f) {
    f = f * 0.5f;  // exact
    e = e + 1;
  }
  float s = (f - 1.0f) / (f + 1.0f);
  float s2 = s * s;
  float p = 0x1.745d18p-4f;  // 1/11
  p = p * s2 + 0x1.c71c72p-4f;  // 1/9
  p = p * s2 + 0x1.24924ap-3f;  // 1/7
  p = p * s2 + 0x1.99999ap-3f;  // 1/5
  p = p * s2 + 0x1.555556p-2f;  // 1/3
  p = p * s2 + 1.0f;
  float ln_f = (2.0f * s) * p;
  return (float)(e - 24) * 0x1.62e430p-1f + ln_f;
}

// The state a reset draws for environment `env` at epoch `epoch`, as the
// binary32 words the state buffers hold: p[3], v[3], q[4] (w, x, y, z).
struct ResetDraw { float p[3], v[3], q[4]; };

inline ResetDraw sample_reset_f32(uint64_t seed, uint32_t env, uint32_t epoch) {
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t w[3][4];
  for (uint32_t slot = 0; slot < 3; ++slot) {
    uint32_t ctr[4] = {env, epoch, slot, 0u};
    philox4x32_10(ctr, key, w[slot]);
  }
  ResetDraw d;
  // position ~ U[-2, 2)^3
  for (int i = 0; i < 3; ++i) d.p[i] = -2.0f + 4.0f * u01_f32(w[0][i]);
  // attitude: axis (rho cos az, rho sin az, z) with z ~ U(-1, 1], az ~ U[0, 2 pi),
  // rotation angle U[0, pi/6), quaternion (cos(a/2), sin(a/2) axis)
  float az = 1.0f - 2.0f * u01_f32(w[0][3]);
  float one_minus = 1.0f - az * az;
  float rho = (one_minus > 0.0f) ? __builtin_sqrtf(one_minus) : 0.0f;
  float ca, sa;
  sincos_turn_f32(w[1][0], &ca, &sa);
  float ax = rho * ca, ay = rho * sa;
  float half = u01_f32(w[1][1]) * 0x1.0c1524p-2f;  // pi/12 in binary32
  float sh, ch;
  sincos_poly_f32(half, &sh, &ch);
  d.q[0] = ch;
  d.q[1] = sh * ax;
  d.q[2] = sh * ay;
  d.q[3] = sh * az;
  // velocity ~ N(0, 0.5^2) by Box-Muller
  float r1 = __builtin_sqrtf(-2.0f * log_u01_f32(w[1][2]));
  float c1, s1;
  sincos_turn_f32(w[1][3], &c1, &s1);
  float r2 = __builtin_sqrtf(-2.0f * log_u01_f32(w[2][0]));
  float c2, s2;
  sincos_turn_f32(w[2][1], &c2, &s2);
  d.v[0] = 0.5f * (r1 * c1);
  d.v[1] = 0.5f * (r1 * s1);
  d.v[2] = 0.5f * (r2 * c2);
  return d;
}

// ---------------------------------------------- obstacle pose re-draw ----
// On a reset the obstacles of the environment may be re-placed (Sec. V: the
// asset manager samples a new position and orientation for every obstacle of
// an environment that resets; position bounds are fractions of the
// environment bounds, orientation bounds are Euler angles, and a dimension
// can be held at a constant value). Box k of environment env at epoch e uses
// two draws: counter (env, e, k, 1) -> x, y, z fractions and roll;
// counter (env, e, k, 2) -> pitch, yaw. Half-extents are kept.
struct BoxRand {
  float pos_min[3], pos_max[3];      // fractions of the environment bounds
  float euler_min[3], euler_max[3];  // roll, pitch, yaw [rad], within [-pi, pi]
  uint32_t lock;                     // bit d: dimension d (x, y, z, roll, pitch, yaw) held at fixed[d]
  float fixed[6];
};

struct BoxPose { float c[3], q[4]; };

inline BoxPose sample_box_pose_f32(uint64_t seed, uint32_t env, uint32_t epoch, uint32_t k, const BoxRand& r,
                                   const float env_min[3], const float env_max[3]) {
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t w1[4], w2[4];
  uint32_t c1[4] = {env, epoch, k, 1u}, c2[4] = {env, epoch, k, 2u};
  philox4x32_10(c1, key, w1);
  philox4x32_10(c2, key, w2);
  BoxPose b;
  for (int d = 0; d < 3; ++d) {
    if (r.lock & (1u << d)) {
      b.c[d] = r.fixed[d];
    } else {
      float f = r.pos_min[d] + (r.pos_max[d] - r.pos_min[d]) * u01_f32(w1[d]);
      b.c[d] = env_min[d] + (env_max[d] - env_min[d]) * f;
    }
  }
  const uint32_t words[3] = {w1[3], w2[0], w2[1]};
  float s[3], c[3];  // sin, cos of the half roll, pitch, yaw
  for (int a = 0; a < 3; ++a) {
    float ang = (r.lock & (1u << (3 + a))) ? r.fixed[3 + a]
                                            : r.euler_min[a] + (r.euler_max[a] - r.euler_min[a]) * u01_f32(words[a]);
    sincos_poly_f32(0.5f * ang, &s[a], &c[a]);
  }
  // q = q_z(yaw) (x) q_y(pitch) (x) q_x(roll)
  const float cr = c[0], sr = s[0], cp = c[1], sp = s[1], cy = c[2], sy = s[2];
  const float cycp = cy * cp, sysp = sy * sp, cysp = cy * sp, sycp = sy * cp;
  b.q[0] = cycp * cr + sysp * sr;
  b.q[1] = cycp * sr - sysp * cr;
  b.q[2] = cysp * cr + sycp * sr;
  b.q[3] = sycp * cr - cysp * sr;
  return b;
}

// Hover thrust per motor written on reset: (m * 9.81) / n_rot in binary32.
inline float hover_thrust_f32(float m, int n_rot) { return (m * 9.81f) / (float)n_rot; }

}  // namespace orc
