// fleet_device.cuh — float32 device math of one multirotor substep.
//
// Everything a thread needs to advance ONE vehicle: the SE(3) geometric
// controller (Kulkarni et al., arXiv 2305.16510, Sec. IV-A Eqs. 1-5, Sec. IV-B
// Eqs. 6-9, and position tracking after Lee, Leok & McClamroch 2011 as
// Sec. I states), rotor allocation with clamp and first-order lag, rigid-body
// derivatives, semi-implicit Euler and RK4 updates, quaternion
// renormalisation and the sphere-vs-oriented-box test.
//
// Differences from the paper's text that change no result beyond float32
// rounding:
//   * the yaw psi = atan2(R10, R00) is never formed: cos psi and sin psi are
//     R00 / rho and R10 / rho with rho = sqrt(R00^2 + R10^2);
//   * Eqs. 8-9 are evaluated without atan2/sin/cos: with a the commanded
//     acceleration, cos(phi_d) = sqrt(a_x^2 + a_z^2) / |a|,
//     sin(phi_d) = -a_y / |a|, cos(theta_d) = a_z / sqrt(a_x^2 + a_z^2),
//     sin(theta_d) = a_x / sqrt(a_x^2 + a_z^2);
//   * R_z(psi) R_y(theta_d) R_x(phi_d) is written out in those cosines and
//     sines, and trig of commanded angles is taken once per launch;
//   * e_R = 1/2 vee(E - E^T) needs only the off-diagonal entries of
//     E = R_d^T R;
//   * Eq. 2 is Omega_d = R_d^T (0, 0, psi_dot_d) (the body rate of a pure
//     world-z yaw rate seen from R_d = R_z R_y R_x), so R_d Omega_d =
//     psi_dot_d e_3 and Eq. 4 becomes e_Omega = Omega - psi_dot_d R^T e_3,
//     i.e. the third row of R times the commanded yaw rate (zero in position
//     mode, where Omega_d = 0);
//   * the first derivative evaluation of a substep reuses the controller's
//     R e_3 (q is unit there: it was renormalised after the last substep);
//   * the body z axis of a non-unit quaternion (RK4 stages 2-4) is the
//     homogeneous quaternion form divided by |q|^2, which equals the axis of
//     q / |q| exactly, and is folded into the stage's acceleration (accel_q);
//   * with the diagonal inertia, Omega x J Omega is written in principal
//     axes, ((Jz - Jy) wy wz, (Jx - Jz) wz wx, (Jy - Jx) wx wy), and J^-1 M is
//     formed once per substep (the wrench is held over the RK4 stages);
//   * the factor 1/2 of q' = 1/2 q (x) (0, Omega) is folded into the RK4
//     stage weights of the quaternion and into the semi-implicit Euler step
//     (multiplications by powers of two are exact);
//   * 1/x and 1/sqrt(x) of squared norms use the hardware approximations
//     (rcp_ftz, rsqrt_ftz), and every fused multiply-add is explicit (the
//     including files are compiled without contraction), so each compiled
//     copy of the step rounds alike.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace agk {

constexpr float kGravity = 9.81f;

enum : int { kModePosition = 0, kModeBodyVel = 1, kModeAttThrust = 2, kModeWrench = 3 };
enum : int { kIntegSIE = 0, kIntegRK4 = 1 };

struct V3 { float x, y, z; };
struct Q4 { float w, x, y, z; };
struct VState { V3 p, v; Q4 q; V3 w; };
struct Wrench4 { float f, mx, my, mz; };
// Rigid-body parameters of one vehicle. With a diagonal inertia the
// gyroscopic term is Omega x J Omega = (gx wy wz, gy wz wx, gz wx wy), where
// (gx, gy, gz) = (Jz - Jy, Jx - Jz, Jy - Jx); (ex, ey, ez) = g / J.
struct Body { float m, inv_m, jx, jy, jz, ijx, ijy, ijz, gx, gy, gz, ex, ey, ez; };

__device__ __forceinline__ Body make_body(float m, float jx, float jy, float jz) {
  Body b;
  b.m = m; b.jx = jx; b.jy = jy; b.jz = jz;
  b.inv_m = 1.f / m; b.ijx = 1.f / jx; b.ijy = 1.f / jy; b.ijz = 1.f / jz;
  b.gx = jz - jy; b.gy = jx - jz; b.gz = jy - jx;
  b.ex = b.gx * b.ijx; b.ey = b.gy * b.ijy; b.ez = b.gz * b.ijz;
  return b;
}

// Gains, rotor matrices and integration constants of one launch; passed by
// value as a kernel parameter (it lives in the constant bank).
struct StepParams {
  float kx[3], kv[3], kR[3], kW[3];
  float A[3][4][8];   // wrench = A u for quad (0), hexa (1), octo (2)
  float Ap[3][8][4];  // pseudo-inverse of A (FP64-computed, stored float32)
  // the same in the pair layout of the packed allocation (pair_rotor_matrices):
  float2 Ap2[3][4][4];  // (Ap[2j][k], Ap[2j + 1][k]): motors 2j and 2j + 1
  float2 A2[3][2][8];   // (A[0][i], A[1][i]) and (A[2][i], A[3][i]): (f, M_x) and (M_y, M_z) of motor i
  float h;            // substep length
  float alpha;        // motor lag factor 1 - exp(-h / tau)
  float drag;
  float r2;           // squared collision radius
  float u_max;
  uint32_t seed_lo, seed_hi;
  uint32_t exact_tests;  // 1: run the collision test at every step (no clearance skip)
};

// Fills the pair layout of the allocation matrices from A and Ap.
inline void pair_rotor_matrices(StepParams& P) {
  for (int t = 0; t < 3; ++t) {
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) P.Ap2[t][j][k] = make_float2(P.Ap[t][2 * j][k], P.Ap[t][2 * j + 1][k]);
    for (int i = 0; i < 8; ++i) {
      P.A2[t][0][i] = make_float2(P.A[t][0][i], P.A[t][1][i]);
      P.A2[t][1][i] = make_float2(P.A[t][2][i], P.A[t][3][i]);
    }
  }
}

__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
// 1/x and 1/sqrt(x) by the hardware approximations with subnormal inputs
// and results flushed to zero (PTX rcp.approx.ftz.f32, rsqrt.approx.ftz.f32).
// Used only where x is a squared norm in the normal range: that of a
// unit-scale quaternion, or one checked against 1e-18 or against the
// smallest normal float (kMinNormal) first; a squared norm below kMinNormal
// counts as 0.
constexpr float kMinNormal = 1.17549435e-38f;  // 2^-126
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x))};
}
// a x b for b = (b.x, b.y, 0)
__device__ __forceinline__ V3 cross_xy(V3 a, float bx, float by) {
  return {-(a.z * by), a.z * bx, fmaf(a.x, by, -(a.y * bx))};
}
__device__ __forceinline__ float dot4(const Q4& q) { return fmaf(q.z, q.z, fmaf(q.y, q.y, fmaf(q.x, q.x, q.w * q.w))); }

// Rotation matrix of a unit quaternion (body -> world), from the doubled
// vector part (doubling is exact): R00 = 1 - 2 y^2 - 2 z^2, R01 = 2 (x y - w z), ...
__device__ __forceinline__ void rotation(const Q4& q, float R[3][3]) {
  const float x2 = 2.f * q.x, y2 = 2.f * q.y, z2 = 2.f * q.z;
  const float wx = q.w * x2, wy = q.w * y2, wz = q.w * z2;
  R[0][0] = fmaf(-q.y, y2, fmaf(-q.z, z2, 1.f));
  R[1][1] = fmaf(-q.x, x2, fmaf(-q.z, z2, 1.f));
  R[2][2] = fmaf(-q.x, x2, fmaf(-q.y, y2, 1.f));
  R[0][1] = fmaf(q.x, y2, -wz); R[1][0] = fmaf(q.x, y2, wz);
  R[0][2] = fmaf(q.x, z2, wy);  R[2][0] = fmaf(q.x, z2, -wy);
  R[1][2] = fmaf(q.y, z2, -wx); R[2][1] = fmaf(q.y, z2, wx);
}

// Per-launch constants of an environment's command. Trig of commanded angles
// is evaluated here once instead of every substep.
//   position:   c = (p_d.x, p_d.y, p_d.z, cos psi_d, sin psi_d, -)
//   body vel:   c = (v_d.x, v_d.y, v_d.z, psi_dot_d, -, -)
//   att+thrust: c = (cos phi_d, sin phi_d, cos theta_d, sin theta_d, psi_dot_d, f)
//   wrench:     c = (f, M_x, M_y, M_z, -, -)
struct Command { int mode; float c[6]; };

__device__ __forceinline__ Command prepare_command(int mode, float t0, float t1, float t2, float t3) {
  Command cm;
  cm.mode = mode > kModeWrench ? kModeWrench : mode;
  cm.c[0] = t0; cm.c[1] = t1; cm.c[2] = t2; cm.c[3] = t3; cm.c[4] = 0.f; cm.c[5] = 0.f;
  if (cm.mode == kModePosition) {
    float s, c;
    sincosf(t3, &s, &c);
    cm.c[3] = c;
    cm.c[4] = s;
  } else if (cm.mode == kModeAttThrust) {
    float sp, cp, st, ct;
    sincosf(t0, &sp, &cp);
    sincosf(t1, &st, &ct);
    cm.c[0] = cp; cm.c[1] = sp; cm.c[2] = ct; cm.c[3] = st; cm.c[4] = t2; cm.c[5] = t3;
  }
  return cm;
}

// Geometric controller of one vehicle -> commanded (f, M). Also returns the
// body z axis R e_3 of the (unit) attitude, which the integrator reuses.
__device__ __forceinline__ Wrench4 controller(const VState& s, const Command& cm, const Body& b,
                                              const StepParams& P, V3& b3) {
  float R[3][3];
  rotation(s.q, R);
  b3 = {R[0][2], R[1][2], R[2][2]};
  if (cm.mode == kModeWrench) return {cm.c[0], cm.c[1], cm.c[2], cm.c[3]};
  float Rd[3][3];
  float rate;  // commanded yaw rate: R_d Omega_d = rate e_3
  float f;
  if (cm.mode == kModePosition) {
    // Lee 2011: a = -k_x e_x - k_v e_v + g e3, b3d = a/|a|, b2d ~ b3d x b1c, b1d = b2d x b3d
    V3 a = {fmaf(-P.kx[0], s.p.x - cm.c[0], -(P.kv[0] * s.v.x)),
            fmaf(-P.kx[1], s.p.y - cm.c[1], -(P.kv[1] * s.v.y)),
            fmaf(-P.kx[2], s.p.z - cm.c[2], fmaf(-P.kv[2], s.v.z, kGravity))};
    f = b.m * dot(a, b3);
    float an2 = dot(a, a);
    V3 b3d = an2 > 1e-18f ? rsqrt_ftz(an2) * a : V3{0.f, 0.f, 1.f};
    V3 c = cross_xy(b3d, cm.c[3], cm.c[4]);  // b1c = (cos psi_d, sin psi_d, 0)
    float cn2 = dot(c, c);
    if (!(cn2 > 1e-18f)) {
      c = cross_xy(b3d, -cm.c[4], cm.c[3]);  // b1c turned by 90 degrees
      cn2 = dot(c, c);
    }
    V3 b2d = rsqrt_ftz(cn2) * c;  // cn2 > 1e-18, or near 1 for the perpendicular heading
    V3 b1d = cross(b2d, b3d);
    Rd[0][0] = b1d.x; Rd[0][1] = b2d.x; Rd[0][2] = b3d.x;
    Rd[1][0] = b1d.y; Rd[1][1] = b2d.y; Rd[1][2] = b3d.y;
    Rd[2][0] = b1d.z; Rd[2][1] = b2d.z; Rd[2][2] = b3d.z;
    rate = 0.f;
  } else {
    // current yaw of the body frame: (cos psi, sin psi) = (R00, R10) / rho
    float rho2 = fmaf(R[1][0], R[1][0], R[0][0] * R[0][0]);
    float cpsi = 1.f, spsi = 0.f;
    if (rho2 >= kMinNormal) {
      float ir = rsqrt_ftz(rho2);
      cpsi = R[0][0] * ir;
      spsi = R[1][0] * ir;
    }
    float cphi, sphi, cth, sth;
    if (cm.mode == kModeBodyVel) {
      // Eq. 6 in the vehicle frame, Eq. 7 thrust, Eqs. 8-9 tilt (algebraic)
      V3 vV = {fmaf(spsi, s.v.y, cpsi * s.v.x), fmaf(cpsi, s.v.y, -(spsi * s.v.x)), s.v.z};
      V3 a = {P.kv[0] * (cm.c[0] - vV.x), P.kv[1] * (cm.c[1] - vV.y), fmaf(P.kv[2], cm.c[2] - vV.z, kGravity)};
      V3 b3V = {fmaf(spsi, R[1][2], cpsi * R[0][2]), fmaf(cpsi, R[1][2], -(spsi * R[0][2])), R[2][2]};
      f = b.m * dot(a, b3V);
      float rxz2 = fmaf(a.z, a.z, a.x * a.x);
      float an2 = fmaf(a.y, a.y, rxz2);
      cphi = 1.f; sphi = 0.f; cth = 1.f; sth = 0.f;
      if (rxz2 >= kMinNormal) {
        float irxz = rsqrt_ftz(rxz2);
        cth = a.z * irxz;
        sth = a.x * irxz;
        float ian = rsqrt_ftz(an2);  // an2 >= rxz2
        cphi = rxz2 * irxz * ian;
        sphi = -a.y * ian;
      } else if (an2 > 0.f) {
        cphi = 0.f;
        sphi = a.y > 0.f ? -1.f : 1.f;
      }
      rate = cm.c[3];
    } else {
      cphi = cm.c[0]; sphi = cm.c[1]; cth = cm.c[2]; sth = cm.c[3]; rate = cm.c[4];
      f = cm.c[5];
    }
    // Eq. 1: R_d = R_z(psi) R_y(theta_d) R_x(phi_d)
    float b01 = sth * sphi, b02 = sth * cphi, b21 = cth * sphi, b22 = cth * cphi;
    Rd[0][0] = cpsi * cth; Rd[0][1] = fmaf(cpsi, b01, -(spsi * cphi)); Rd[0][2] = fmaf(cpsi, b02, spsi * sphi);
    Rd[1][0] = spsi * cth; Rd[1][1] = fmaf(spsi, b01, cpsi * cphi);    Rd[1][2] = fmaf(spsi, b02, -(cpsi * sphi));
    Rd[2][0] = -sth;       Rd[2][1] = b21;                             Rd[2][2] = b22;
  }
  // Eq. 3: e_R = 1/2 vee(E - E^T), E = R_d^T R (off-diagonal entries only); each component is
  // E_ij - E_ji = col_i(R_d) . col_j(R) - col_j(R_d) . col_i(R) as one chain of six products, and
  // its factor 1/2 is exact, so it is applied with the gain below
  auto dE = [&](int i, int j) {
    return fmaf(Rd[0][i], R[0][j], fmaf(Rd[1][i], R[1][j], fmaf(Rd[2][i], R[2][j],
           fmaf(-Rd[0][j], R[0][i], fmaf(-Rd[1][j], R[1][i], -(Rd[2][j] * R[2][i]))))));
  };
  const V3 eR2 = {dE(2, 1), dE(0, 2), dE(1, 0)};  // 2 e_R
  // Eq. 4 with R^T R_d Omega_d = rate R^T e_3
  V3 eW = {fmaf(-rate, R[2][0], s.w.x), fmaf(-rate, R[2][1], s.w.y), fmaf(-rate, R[2][2], s.w.z)};
  // Eq. 5's Omega x J Omega in principal axes
  const V3 gyro = {b.gx * (s.w.y * s.w.z), b.gy * (s.w.z * s.w.x), b.gz * (s.w.x * s.w.y)};
  return {f, fmaf(-0.5f * P.kR[0], eR2.x, fmaf(-P.kW[0], eW.x, gyro.x)),
          fmaf(-0.5f * P.kR[1], eR2.y, fmaf(-P.kW[1], eW.y, gyro.y)),
          fmaf(-0.5f * P.kR[2], eR2.z, fmaf(-P.kW[2], eW.z, gyro.z))};
}

// Rotor allocation, per-motor clamp to [0, u_max], first-order lag; returns
// the realised wrench A u. Two motors travel as one FP32 pair through the
// allocation and the lag, and the wrench accumulates as the pairs (f, M_x)
// and (M_y, M_z), in packed FMAs (__ffma2_rn) that round each lane as the
// scalar form would, in the same order.
template <int NROT>
__device__ __forceinline__ Wrench4 allocate(const Wrench4& cmd, float (&u)[NROT], const StepParams& P) {
  constexpr int T = NROT == 4 ? 0 : (NROT == 6 ? 1 : 2);
  const float2 f2 = make_float2(cmd.f, cmd.f), mx2 = make_float2(cmd.mx, cmd.mx);
  const float2 my2 = make_float2(cmd.my, cmd.my), mz2 = make_float2(cmd.mz, cmd.mz);
  const float2 alpha2 = make_float2(P.alpha, P.alpha);
  float2 Wa = make_float2(0.f, 0.f), Wb = make_float2(0.f, 0.f);  // (f, M_x), (M_y, M_z)
#pragma unroll
  for (int j = 0; j < NROT / 2; ++j) {
    float2 uc = __ffma2_rn(P.Ap2[T][j][3], mz2,
                           __ffma2_rn(P.Ap2[T][j][2], my2, __ffma2_rn(P.Ap2[T][j][1], mx2, __fmul2_rn(P.Ap2[T][j][0], f2))));
    uc = make_float2(fminf(fmaxf(uc.x, 0.f), P.u_max), fminf(fmaxf(uc.y, 0.f), P.u_max));
    float2 uu = make_float2(u[2 * j], u[2 * j + 1]);
    uu = __ffma2_rn(alpha2, __fadd2_rn(uc, make_float2(-uu.x, -uu.y)), uu);
    u[2 * j] = uu.x;
    u[2 * j + 1] = uu.y;
    const float2 u0 = make_float2(uu.x, uu.x), u1 = make_float2(uu.y, uu.y);
    Wa = __ffma2_rn(P.A2[T][0][2 * j], u0, Wa);
    Wb = __ffma2_rn(P.A2[T][1][2 * j], u0, Wb);
    Wa = __ffma2_rn(P.A2[T][0][2 * j + 1], u1, Wa);
    Wb = __ffma2_rn(P.A2[T][1][2 * j + 1], u1, Wb);
  }
  return {Wa.x, Wa.y, Wb.x, Wb.y};
}

// Body z axis of a possibly non-unit quaternion: the homogeneous form over
// |q|^2, 2 (xz + wy, yz - wx, .) / |q|^2, with its third component written
// as 1 - 2 (x^2 + y^2) / |q|^2 (w^2 + z^2 = |q|^2 - x^2 - y^2).
__device__ __forceinline__ V3 body_z(const Q4& q) {
  const float inv2 = 2.f * rcp_ftz(dot4(q));
  return {inv2 * fmaf(q.x, q.z, q.w * q.y), inv2 * fmaf(q.y, q.z, -(q.w * q.x)),
          fmaf(-inv2, fmaf(q.x, q.x, q.y * q.y), 1.f)};
}

__device__ __forceinline__ void normalize(Q4& q) {
  float r = rsqrt_ftz(dot4(q));
  q.w *= r; q.x *= r; q.y *= r; q.z *= r;
}

// q (x) (0, w): twice the quaternion rate q' = 1/2 q (x) (0, Omega)
__device__ __forceinline__ Q4 quat_rate2(const Q4& q, const V3& w) {
  return {-fmaf(q.z, w.z, fmaf(q.y, w.y, q.x * w.x)), fmaf(q.w, w.x, fmaf(q.y, w.z, -(q.z * w.y))),
          fmaf(q.w, w.y, fmaf(q.z, w.x, -(q.x * w.z))), fmaf(q.w, w.z, fmaf(q.x, w.y, -(q.y * w.x)))};
}

// The rigid-body rates under the wrench held over a substep:
//   v' = fm b3 - (c/m) v + g,  Omega' = J^-1 M - e (wy wz, wz wx, wx wy)
// with fm = f / m and aw = J^-1 M computed once per substep (Euler's
// equations in principal axes).
template <bool DRAG>
__device__ __forceinline__ V3 accel(V3 b3, V3 v, float fm, float dm) {
  if (DRAG)
    return {fmaf(fm, b3.x, -(dm * v.x)), fmaf(fm, b3.y, -(dm * v.y)), fmaf(fm, b3.z, fmaf(-dm, v.z, -kGravity))};
  return {fm * b3.x, fm * b3.y, fmaf(fm, b3.z, -kGravity)};
}

// v' of an RK4 stage whose quaternion q need not be unit, with the body z
// axis b3(q) = (2 (xz + wy), 2 (yz - wx), |q|^2 - 2 (x^2 + y^2)) / |q|^2
// folded in: with s = 2 fm / |q|^2, v' = (s (xz + wy), s (yz - wx),
// (fm - g) - s (x^2 + y^2)) - (c/m) v. fm2 = 2 fm and fmg = fm - g are taken
// once per substep.
template <bool DRAG>
__device__ __forceinline__ V3 accel_q(const Q4& q, V3 v, float fm2, float fmg, float dm) {
  const float s = fm2 * rcp_ftz(dot4(q));
  const float px = fmaf(q.x, q.z, q.w * q.y), py = fmaf(q.y, q.z, -(q.w * q.x)), pz = fmaf(q.x, q.x, q.y * q.y);
  if (DRAG) return {fmaf(s, px, -(dm * v.x)), fmaf(s, py, -(dm * v.y)), fmaf(-s, pz, fmaf(-dm, v.z, fmg))};
  return {s * px, s * py, fmaf(-s, pz, fmg)};
}

__device__ __forceinline__ V3 ang_accel(V3 w, V3 aw, const Body& b) {
  return {fmaf(-b.ex, w.y * w.z, aw.x), fmaf(-b.ey, w.z * w.x, aw.y), fmaf(-b.ez, w.x * w.y, aw.z)};
}

// Semi-implicit Euler: v, Omega from the rates; p, q from the updated
// velocities; renormalise q. b3 is R e_3 of the (unit) start attitude.
template <bool DRAG>
__device__ __forceinline__ void step_sie(VState& s, V3 b3, const Wrench4& W, const Body& b, float drag, float h) {
  const float fm = W.f * b.inv_m, dm = drag * b.inv_m;
  const V3 aw = {b.ijx * W.mx, b.ijy * W.my, b.ijz * W.mz};
  const V3 dv = accel<DRAG>(b3, s.v, fm, dm);
  const V3 dw = ang_accel(s.w, aw, b);
  // the updates as FP32 pairs (v_x v_y) (v_z w_x) (w_y w_z) (p_x p_y) (q_w q_x) (q_y q_z), each lane
  // rounded as the scalar fmaf
  const float2 h2 = make_float2(h, h);
  const float2 vxy = __ffma2_rn(h2, make_float2(dv.x, dv.y), make_float2(s.v.x, s.v.y));
  const float2 vzwx = __ffma2_rn(h2, make_float2(dv.z, dw.x), make_float2(s.v.z, s.w.x));
  const float2 wyz = __ffma2_rn(h2, make_float2(dw.y, dw.z), make_float2(s.w.y, s.w.z));
  s.v = {vxy.x, vxy.y, vzwx.x};
  s.w = {vzwx.y, wyz.x, wyz.y};
  const float2 pxy = __ffma2_rn(h2, vxy, make_float2(s.p.x, s.p.y));
  s.p = {pxy.x, pxy.y, fmaf(h, s.v.z, s.p.z)};
  const float hh = 0.5f * h;
  const float2 hh2 = make_float2(hh, hh);
  const Q4 r = quat_rate2(s.q, s.w);
  const float2 qwx = __ffma2_rn(hh2, make_float2(r.w, r.x), make_float2(s.q.w, s.q.x));
  const float2 qyz = __ffma2_rn(hh2, make_float2(r.y, r.z), make_float2(s.q.y, s.q.z));
  s.q = {qwx.x, qwx.y, qyz.x, qyz.y};
  normalize(s.q);
}

// Classic RK4 on (p, v, q, Omega) with the wrench held over the stages;
// renormalise q. The first stage uses the start attitude's b3 (unit q), the
// others the body z axis of their stage quaternion (accel_q).
//
// The state travels as seven FP32 pairs, (vx vy) (vz wx) (wy wz) (qw qx)
// (qy qz) (px py) (pz -), and each stage's rates in the same order as
// (v' | Omega' | 2 q' | p'), with 2 q' = q (x) (0, Omega): the quaternion's
// factor 1/2 goes into its pairs' stage and step weights instead. Every
// stage state x + c k and every accumulation s + 2 k is then one packed FMA
// per pair (__ffma2_rn); halving a weight is exact, so each product equals
// that of the scalar form.
// The rates of stage state y given its v' (a).
__device__ __forceinline__ void rk4_rates(const float2 (&y)[7], V3 a, V3 aw, const Body& b, float2 (&k)[7]) {
  const V3 v = {y[0].x, y[0].y, y[1].x}, w = {y[1].y, y[2].x, y[2].y};
  const Q4 q = {y[3].x, y[3].y, y[4].x, y[4].y};
  const V3 al = ang_accel(w, aw, b);
  const Q4 r = quat_rate2(q, w);  // twice the quaternion rate
  k[0] = make_float2(a.x, a.y);
  k[1] = make_float2(a.z, al.x);
  k[2] = make_float2(al.y, al.z);
  k[3] = make_float2(r.w, r.x);
  k[4] = make_float2(r.y, r.z);
  k[5] = make_float2(v.x, v.y);
  k[6] = make_float2(v.z, 0.f);
}

template <bool DRAG>
__device__ __forceinline__ void step_rk4(VState& s, V3 b3, const Wrench4& W, const Body& b, float drag, float h) {
  const float fm = W.f * b.inv_m, dm = drag * b.inv_m;
  const V3 aw = {b.ijx * W.mx, b.ijy * W.my, b.ijz * W.mz};
  const float2 x[7] = {make_float2(s.v.x, s.v.y), make_float2(s.v.z, s.w.x), make_float2(s.w.y, s.w.z),
                       make_float2(s.q.w, s.q.x), make_float2(s.q.y, s.q.z), make_float2(s.p.x, s.p.y),
                       make_float2(s.p.z, 0.f)};
  float2 k[7], acc[7], y[7];
  // stage 1; acc collects k1 + 2 k2 + 2 k3 + k4
  rk4_rates(x, accel<DRAG>(b3, s.v, fm, dm), aw, b, k);
#pragma unroll
  for (int i = 0; i < 7; ++i) acc[i] = k[i];
  // stages 2 and 3 at t + h/2, stage 4 at t + h, each from the previous stage's rates
  const float fm2 = 2.f * fm, fmg = fm - kGravity;
  const float2 c2 = make_float2(0.5f * h, 0.5f * h), c4 = make_float2(h, h), two = make_float2(2.f, 2.f);
  const float2 c2q = make_float2(0.25f * h, 0.25f * h), c4q = make_float2(0.5f * h, 0.5f * h);
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const float2 c = st < 2 ? c2 : c4, cq = st < 2 ? c2q : c4q;
#pragma unroll
    for (int i = 0; i < 5; ++i) y[i] = __ffma2_rn(i >= 3 ? cq : c, k[i], x[i]);  // v, Omega, q (p is not needed)
    rk4_rates(y, accel_q<DRAG>({y[3].x, y[3].y, y[4].x, y[4].y}, {y[0].x, y[0].y, y[1].x}, fm2, fmg, dm), aw, b, k);
#pragma unroll
    for (int i = 0; i < 7; ++i) acc[i] = st < 2 ? __ffma2_rn(two, k[i], acc[i]) : __fadd2_rn(k[i], acc[i]);
  }
  // x + h/6 (k1 + 2 k2 + 2 k3 + k4)
  const float h6 = h * (1.f / 6.f);
  const float2 c6 = make_float2(h6, h6), c6q = make_float2(0.5f * h6, 0.5f * h6);
  float2 xn[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) xn[i] = __ffma2_rn(i == 3 || i == 4 ? c6q : c6, acc[i], x[i]);
  s.v = {xn[0].x, xn[0].y, xn[1].x};
  s.w = {xn[1].y, xn[2].x, xn[2].y};
  s.q = {xn[3].x, xn[3].y, xn[4].x, xn[4].y};
  s.p = {xn[5].x, xn[5].y, xn[6].x};
  normalize(s.q);
}

template <int INTEG, bool DRAG>
__device__ __forceinline__ void integrate(VState& s, V3 b3, const Wrench4& W, const Body& b, const StepParams& P) {
  if (INTEG == kIntegRK4)
    step_rk4<DRAG>(s, b3, W, b, P.drag, P.h);
  else
    step_sie<DRAG>(s, b3, W, b, P.drag, P.h);
}

// Sphere of squared radius r2 at p versus the box (centre c, half-extents
// hx, hy, hz, unit quaternion qb): p is taken into the box frame by the
// conjugate rotation v - w t + u x t with t = 2 u x v; the distance to the
// box is the norm of max(|d| - h, 0) per axis (equal to |d - clamp(d, -h, h)|);
// touching counts. The operations and their order are those of the fused
// step's paired test (pair_dist2), so both take the same decisions.
__device__ __forceinline__ bool sphere_hits_box(V3 p, float r2, V3 c, V3 hb, Q4 qb) {
  const V3 v = p - c;
  const V3 u2 = {2.f * qb.x, 2.f * qb.y, 2.f * qb.z};
  const V3 t = cross(u2, v);                  // 2 u x v
  const V3 ut2 = cross(u2, t);                // 2 (u x t)
  const V3 d = {fmaf(0.5f, ut2.x, fmaf(-qb.w, t.x, v.x)), fmaf(0.5f, ut2.y, fmaf(-qb.w, t.y, v.y)),
                fmaf(0.5f, ut2.z, fmaf(-qb.w, t.z, v.z))};
  const float ex = fmaxf(fabsf(d.x) - hb.x, 0.f);
  const float ey = fmaxf(fabsf(d.y) - hb.y, 0.f);
  const float ez = fmaxf(fabsf(d.z) - hb.z, 0.f);
  return !(r2 < fmaf(ez, ez, fmaf(ey, ey, ex * ex)));
}

}  // namespace agk
