// aerial_oracle.hpp — plain FP64 CPU oracle of the multirotor fleet step.
//
// TEST INFRASTRUCTURE ONLY. This is the slow, obviously-correct reference
// that the CUDA path is checked against. Only tests/, __graft_entry__.smoke()
// and the cpu_baseline / reference legs of bench.py load it. The product
// library never links, loads or calls it, and it shares no code, header,
// constant or table with the CUDA sources.
//
// What it follows (Kulkarni, Forgaard, Alexis, "Aerial Gym - Isaac Gym
// Simulator for Aerial Robots", arXiv 2305.16510):
//   * Sec. IV-A, Eqs. 1-5: attitude-controlled flight mode (desired frame,
//     desired body rate, attitude and rate errors, moment law with the
//     gyroscopic feed-forward term kept).
//   * Sec. IV-B, Eqs. 6-9: velocity-controlled flight mode in the yaw-aligned
//     vehicle frame V.
//   * Sec. I (position tracking in the inertial frame) with the construction
//     of Lee, Leok & McClamroch 2011 (the paper's basis, ref. [lee2011control]).
//   * Sec. I / IV-B last sentence: force and torque applied to a rigid body;
//     the 6-DoF dynamics, rotor allocation, motor lag, collision and reset
//     are the readings listed in each function's comment.
//   * Sec. III (depth cameras) and Sec. I / VII (kernel-based ray casting):
//     ray_box_depth, the slab method for a pinhole camera's rays.
//   * Sec. V (obstacle poses re-drawn on reset): philox_sampler.hpp.
//   * Sec. I (learning to reach a goal setpoint): the task's observation,
//     reward and termination in oracle_capi.cpp (orc_reach_task).
//
// Every function is a template on the scalar type T so the same code runs
// in double (the oracle), in an op-counting scalar (algorithmic FLOPs per
// vehicle-step) and in a forward-mode dual number (JVP checks of the
// adjoint). The reset sampler is the one exception: it is defined in strict
// IEEE FP32 (see philox_sampler.hpp) and its words are widened to T.
#pragma once

#include <cmath>
#include <cstdint>

namespace orc {

// ---------------------------------------------------------------- vectors --
template <class T> struct Vec3 { T x, y, z; };
template <class T> struct Mat3 { T a[3][3]; };  // row-major, a[row][col]
template <class T> struct Quat { T w, x, y, z; };  // Hamilton, body -> world

template <class T> Vec3<T> operator+(Vec3<T> a, Vec3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> Vec3<T> operator-(Vec3<T> a, Vec3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> Vec3<T> operator-(Vec3<T> a) { return {-a.x, -a.y, -a.z}; }
template <class T> Vec3<T> scale(T s, Vec3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
// element-wise product: diagonal gain or diagonal inertia times a vector
template <class T> Vec3<T> diag_mul(Vec3<T> d, Vec3<T> a) { return {d.x * a.x, d.y * a.y, d.z * a.z}; }
template <class T> T dot(Vec3<T> a, Vec3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> Vec3<T> cross(Vec3<T> a, Vec3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> T norm(Vec3<T> a) { using std::sqrt; return sqrt(dot(a, a)); }

template <class T> Mat3<T> transpose(const Mat3<T>& m) {
  Mat3<T> t;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t.a[i][j] = m.a[j][i];
  return t;
}
template <class T> Mat3<T> matmul(const Mat3<T>& m, const Mat3<T>& n) {
  Mat3<T> r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.a[i][j] = m.a[i][0] * n.a[0][j] + m.a[i][1] * n.a[1][j] + m.a[i][2] * n.a[2][j];
  return r;
}
template <class T> Vec3<T> matvec(const Mat3<T>& m, Vec3<T> v) {
  return {m.a[0][0] * v.x + m.a[0][1] * v.y + m.a[0][2] * v.z,
          m.a[1][0] * v.x + m.a[1][1] * v.y + m.a[1][2] * v.z,
          m.a[2][0] * v.x + m.a[2][1] * v.y + m.a[2][2] * v.z};
}
template <class T> Vec3<T> column(const Mat3<T>& m, int j) { return {m.a[0][j], m.a[1][j], m.a[2][j]}; }
template <class T> Mat3<T> from_columns(Vec3<T> c0, Vec3<T> c1, Vec3<T> c2) {
  Mat3<T> m;
  m.a[0][0] = c0.x; m.a[1][0] = c0.y; m.a[2][0] = c0.z;
  m.a[0][1] = c1.x; m.a[1][1] = c1.y; m.a[2][1] = c1.z;
  m.a[0][2] = c2.x; m.a[1][2] = c2.y; m.a[2][2] = c2.z;
  return m;
}

// hat map R^3 -> so(3): hat(a) b = a x b.
template <class T> Mat3<T> hat(Vec3<T> a) {
  Mat3<T> m;
  m.a[0][0] = T(0);  m.a[0][1] = -a.z;  m.a[0][2] = a.y;
  m.a[1][0] = a.z;   m.a[1][1] = T(0);  m.a[1][2] = -a.x;
  m.a[2][0] = -a.y;  m.a[2][1] = a.x;   m.a[2][2] = T(0);
  return m;
}
// vee map so(3) -> R^3, the inverse of hat (Eq. 3's "vee").
template <class T> Vec3<T> vee(const Mat3<T>& m) { return {m.a[2][1], m.a[0][2], m.a[1][0]}; }

// Elementary rotations R_x, R_y, R_z by an angle in radians (Eq. 1; the
// paper's "degrees" is read as radians).
template <class T> Mat3<T> rot_x(T ang) {
  using std::cos; using std::sin;
  T c = cos(ang), s = sin(ang);
  Mat3<T> m;
  m.a[0][0] = T(1); m.a[0][1] = T(0); m.a[0][2] = T(0);
  m.a[1][0] = T(0); m.a[1][1] = c;    m.a[1][2] = -s;
  m.a[2][0] = T(0); m.a[2][1] = s;    m.a[2][2] = c;
  return m;
}
template <class T> Mat3<T> rot_y(T ang) {
  using std::cos; using std::sin;
  T c = cos(ang), s = sin(ang);
  Mat3<T> m;
  m.a[0][0] = c;    m.a[0][1] = T(0); m.a[0][2] = s;
  m.a[1][0] = T(0); m.a[1][1] = T(1); m.a[1][2] = T(0);
  m.a[2][0] = -s;   m.a[2][1] = T(0); m.a[2][2] = c;
  return m;
}
template <class T> Mat3<T> rot_z(T ang) {
  using std::cos; using std::sin;
  T c = cos(ang), s = sin(ang);
  Mat3<T> m;
  m.a[0][0] = c;    m.a[0][1] = -s;   m.a[0][2] = T(0);
  m.a[1][0] = s;    m.a[1][1] = c;    m.a[1][2] = T(0);
  m.a[2][0] = T(0); m.a[2][1] = T(0); m.a[2][2] = T(1);
  return m;
}

template <class T> Quat<T> quat_mul(Quat<T> a, Quat<T> b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
          a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
          a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
template <class T> Quat<T> quat_normalize(Quat<T> q) {
  using std::sqrt;
  T n = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return {q.w / n, q.x / n, q.y / n, q.z / n};
}
// Rotation matrix of the orientation a (not necessarily unit) quaternion
// represents: the standard unit-quaternion formula applied to q / |q|.
// This is the body -> world rotation R of Sec. IV.
template <class T> Mat3<T> quat_to_rot(Quat<T> q_in) {
  Quat<T> q = quat_normalize(q_in);
  T w = q.w, x = q.x, y = q.y, z = q.z;
  Mat3<T> m;
  m.a[0][0] = T(1) - T(2) * (y * y + z * z);
  m.a[0][1] = T(2) * (x * y - w * z);
  m.a[0][2] = T(2) * (x * z + w * y);
  m.a[1][0] = T(2) * (x * y + w * z);
  m.a[1][1] = T(1) - T(2) * (x * x + z * z);
  m.a[1][2] = T(2) * (y * z - w * x);
  m.a[2][0] = T(2) * (x * z - w * y);
  m.a[2][1] = T(2) * (y * z + w * x);
  m.a[2][2] = T(1) - T(2) * (x * x + y * y);
  return m;
}

// Third column of quat_to_rot(q): the body z axis b_3 in the world frame.
template <class T> Vec3<T> body_z_axis(Quat<T> q_in) {
  Quat<T> q = quat_normalize(q_in);
  return {T(2) * (q.x * q.z + q.w * q.y), T(2) * (q.y * q.z - q.w * q.x), T(1) - T(2) * (q.x * q.x + q.y * q.y)};
}

// Rotation matrix of a quaternion that is already unit (box orientations are
// given as unit quaternions and used as they are).
template <class T> Mat3<T> unit_quat_to_rot(Quat<T> q) {
  T w = q.w, x = q.x, y = q.y, z = q.z;
  Mat3<T> m;
  m.a[0][0] = T(1) - T(2) * (y * y + z * z);
  m.a[0][1] = T(2) * (x * y - w * z);
  m.a[0][2] = T(2) * (x * z + w * y);
  m.a[1][0] = T(2) * (x * y + w * z);
  m.a[1][1] = T(1) - T(2) * (x * x + z * z);
  m.a[1][2] = T(2) * (y * z - w * x);
  m.a[2][0] = T(2) * (x * z - w * y);
  m.a[2][1] = T(2) * (y * z + w * x);
  m.a[2][2] = T(1) - T(2) * (x * x + y * y);
  return m;
}

template <class T> T clamp(T v, T lo, T hi) {
  if (v < lo) return lo;
  if (hi < v) return hi;
  return v;
}

// ------------------------------------------------------------- parameters --
constexpr double kGravity = 9.81;  // |g| in m/s^2; g = (0, 0, -9.81), z up

enum Mode : int { MODE_POSITION = 0, MODE_BODY_VEL = 1, MODE_ATT_THRUST = 2, MODE_WRENCH = 3 };

template <class T> struct Gains { Vec3<T> kx, kv, kR, kW; };  // diagonal gain matrices

template <class T> struct Body {  // per-environment rigid-body parameters
  T m;         // total mass [kg]
  Vec3<T> J;   // diagonal of the body-frame inertia [kg m^2]
};

template <class T> struct State {
  Vec3<T> p;   // position of the centre of mass, world frame [m]
  Vec3<T> v;   // velocity of the centre of mass, world frame [m/s]
  Quat<T> q;   // attitude, body -> world
  Vec3<T> w;   // angular velocity Omega, body frame [rad/s]
};

template <class T> struct Wrench {
  T f;         // collective thrust along +b3 [N]
  Vec3<T> M;   // moment, body frame [N m]
};

// Output of the geometric controller for one vehicle at one substep.
template <class T> struct ControlOut {
  Wrench<T> cmd;  // commanded thrust f and moment M (Eq. 5 / Eq. 7)
  Mat3<T> Rd;     // desired body -> world rotation
  Vec3<T> Wd;     // desired body rate Omega_d (Eq. 2)
  Vec3<T> eR;     // attitude error (Eq. 3)
  Vec3<T> eW;     // rate error (Eq. 4)
};

// ------------------------------------------------------------- controller --
// Attitude and rate errors and the moment law, Sec. IV-A Eqs. 3-5:
//   e_R = 1/2 (R_d^T R - R^T R_d)^vee,   e_Omega = Omega - R^T R_d Omega_d,
//   M = -k_R e_R - k_Omega e_Omega + Omega x J Omega.
// R^T R_d is the transpose of R_d^T R, so one product E = R_d^T R serves both.
template <class T>
void attitude_law(const Mat3<T>& R, Vec3<T> W, const Mat3<T>& Rd, Vec3<T> Wd, const Body<T>& body,
                  const Gains<T>& g, ControlOut<T>& out) {
  Mat3<T> E = matmul(transpose(Rd), R);  // R_d^T R
  Mat3<T> Et = transpose(E);             // R^T R_d
  Mat3<T> skew;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) skew.a[i][j] = E.a[i][j] - Et.a[i][j];
  out.eR = scale(T(0.5), vee(skew));
  out.eW = W - matvec(Et, Wd);
  Vec3<T> JW = diag_mul(body.J, W);
  out.cmd.M = -diag_mul(g.kR, out.eR) - diag_mul(g.kW, out.eW) + cross(W, JW);
  out.Rd = Rd;
  out.Wd = Wd;
}

// Current yaw psi of the body frame, read as the Z-Y-X Euler yaw:
// psi = atan2(R_10, R_00) (Sec. IV "the current yaw angle of the robot").
template <class T> T current_yaw(const Mat3<T>& R) {
  using std::atan2;
  return atan2(R.a[1][0], R.a[0][0]);
}

// Eq. 2: desired body rate from a commanded yaw rate at reference roll phi_d
// and pitch theta_d.
template <class T> Vec3<T> desired_rate(T phi_d, T theta_d, T yaw_rate_d) {
  using std::cos; using std::sin;
  Mat3<T> E;
  E.a[0][0] = T(1); E.a[0][1] = T(0);          E.a[0][2] = -sin(theta_d);
  E.a[1][0] = T(0); E.a[1][1] = cos(phi_d);    E.a[1][2] = sin(phi_d) * cos(theta_d);
  E.a[2][0] = T(0); E.a[2][1] = -sin(phi_d);   E.a[2][2] = cos(phi_d) * cos(theta_d);
  Vec3<T> r = {T(0), T(0), yaw_rate_d};
  return matvec(E, r);
}

// Attitude-controlled flight mode, Sec. IV-A: commands (phi_d, theta_d,
// psi_dot_d, f). Eq. 1: R_d = R_z(psi) R_y(theta_d) R_x(phi_d) with psi the
// current yaw; Eq. 2 for Omega_d; Eqs. 3-5 for M. f is the commanded
// collective thrust in newtons.
template <class T>
ControlOut<T> control_attitude(const State<T>& s, T phi_d, T theta_d, T yaw_rate_d, T f_cmd,
                               const Body<T>& body, const Gains<T>& g) {
  Mat3<T> R = quat_to_rot(s.q);
  T psi = current_yaw(R);
  Mat3<T> Rd = matmul(rot_z(psi), matmul(rot_y(theta_d), rot_x(phi_d)));
  ControlOut<T> out;
  attitude_law(R, s.w, Rd, desired_rate(phi_d, theta_d, yaw_rate_d), body, g, out);
  out.cmd.f = f_cmd;
  return out;
}

// Velocity-controlled flight mode, Sec. IV-B, Eqs. 6-9, in the vehicle frame
// V = R_z(psi):
//   v^V = R_z(psi)^T v,   a = k_v (v_d - v^V) + |g| e_3          (Eq. 6)
//   f   = m a . (R_z(psi)^T b_3)                                 (Eq. 7)
//   phi_d = atan2(-a_y, sqrt(a_x^2 + a_z^2)), theta_d = atan2(a_x, a_z)
//                                                               (Eqs. 8-9)
// then Eqs. 1-5 with the commanded yaw rate. Reading: Eq. 7's "(a_d + m g)"
// mixes an acceleration and a force; it is read as m (a_d + |g| e_3), and the
// tilt angles use the same a (with a_d alone, hover would give atan2(0, 0)).
template <class T>
ControlOut<T> control_velocity(const State<T>& s, Vec3<T> v_d, T yaw_rate_d, const Body<T>& body,
                               const Gains<T>& g) {
  using std::atan2; using std::sqrt;
  Mat3<T> R = quat_to_rot(s.q);
  T psi = current_yaw(R);
  Mat3<T> Rpsi = rot_z(psi);
  Vec3<T> vV = matvec(transpose(Rpsi), s.v);
  Vec3<T> a = diag_mul(g.kv, v_d - vV) + Vec3<T>{T(0), T(0), T(kGravity)};
  T phi_d = atan2(-a.y, sqrt(a.x * a.x + a.z * a.z));
  T theta_d = atan2(a.x, a.z);
  Vec3<T> b3_V = matvec(transpose(Rpsi), column(R, 2));
  Mat3<T> Rd = matmul(Rpsi, matmul(rot_y(theta_d), rot_x(phi_d)));
  ControlOut<T> out;
  attitude_law(R, s.w, Rd, desired_rate(phi_d, theta_d, yaw_rate_d), body, g, out);
  out.cmd.f = body.m * dot(a, b3_V);
  return out;
}

// Position tracking in the inertial frame (Sec. I; the paper's controller is
// built on Lee, Leok & McClamroch 2011). Reading, with acceleration-level
// gains so the same k_x, k_v serve every mass:
//   e_x = p - p_d, e_v = v,  a = -k_x e_x - k_v e_v + |g| e_3,
//   f = m a . b_3,  b_3d = a / |a|,  b_1c = (cos psi_d, sin psi_d, 0),
//   b_2d = (b_3d x b_1c) / |b_3d x b_1c|,  b_1d = b_2d x b_3d,
//   R_d = [b_1d b_2d b_3d],  Omega_d = 0
// (the Omega_d feed-forward is dropped the way Sec. IV-A drops Lee's last
// moment term). Degenerate directions (|a| = 0, a parallel to b_1c) fall back
// to b_3d = e_3 and to b_1c rotated by 90 degrees.
template <class T>
ControlOut<T> control_position(const State<T>& s, Vec3<T> p_d, T yaw_d, const Body<T>& body,
                               const Gains<T>& g) {
  using std::cos; using std::sin;
  Mat3<T> R = quat_to_rot(s.q);
  Vec3<T> ex = s.p - p_d;
  Vec3<T> ev = s.v;
  Vec3<T> a = -diag_mul(g.kx, ex) - diag_mul(g.kv, ev) + Vec3<T>{T(0), T(0), T(kGravity)};
  T an = norm(a);
  Vec3<T> b3d = (an > T(1e-9)) ? scale(T(1) / an, a) : Vec3<T>{T(0), T(0), T(1)};
  Vec3<T> b1c = {cos(yaw_d), sin(yaw_d), T(0)};
  Vec3<T> c = cross(b3d, b1c);
  T cn = norm(c);
  if (!(cn > T(1e-9))) {
    b1c = {-sin(yaw_d), cos(yaw_d), T(0)};
    c = cross(b3d, b1c);
    cn = norm(c);
  }
  Vec3<T> b2d = scale(T(1) / cn, c);
  Vec3<T> b1d = cross(b2d, b3d);
  Mat3<T> Rd = from_columns(b1d, b2d, b3d);
  ControlOut<T> out;
  attitude_law(R, s.w, Rd, Vec3<T>{T(0), T(0), T(0)}, body, g, out);
  out.cmd.f = body.m * dot(a, column(R, 2));
  return out;
}

// Commanded target of one environment: mode plus four numbers.
//   POSITION:   (p_d.x, p_d.y, p_d.z, psi_d)
//   BODY_VEL:   (v_d.x, v_d.y, v_d.z, psi_dot_d)   (v_d in frame V)
//   ATT_THRUST: (phi_d, theta_d, psi_dot_d, f)
//   WRENCH:     (f, M_x, M_y, M_z)                 (bypasses the controller)
template <class T>
Wrench<T> controller(int mode, const State<T>& s, const T tgt[4], const Body<T>& body, const Gains<T>& g,
                     ControlOut<T>* detail = nullptr) {
  ControlOut<T> out;
  switch (mode) {
    case MODE_POSITION:
      out = control_position(s, Vec3<T>{tgt[0], tgt[1], tgt[2]}, tgt[3], body, g);
      break;
    case MODE_BODY_VEL:
      out = control_velocity(s, Vec3<T>{tgt[0], tgt[1], tgt[2]}, tgt[3], body, g);
      break;
    case MODE_ATT_THRUST:
      out = control_attitude(s, tgt[0], tgt[1], tgt[2], tgt[3], body, g);
      break;
    default:
      out.cmd.f = tgt[0];
      out.cmd.M = {tgt[1], tgt[2], tgt[3]};
      break;
  }
  if (detail) *detail = out;
  return out.cmd;
}

// ------------------------------------------------------- rotor allocation --
// Reading (the paper only says motor torque must not be ignored, Sec. II):
// n_rot rotors in the body x-y plane at radius `arm`, rotor i at angle
// beta_i = beta_0 + i * 360/n_rot degrees (beta_0 = 45 quad "X", 30 hexa,
// 22.5 octo), thrust u_i along +b_3, reaction torque s_i * k_yaw * u_i about
// b_3 with s_i = +1, -1, +1, ... . The allocation matrix maps rotor thrusts
// to the body wrench W = (f, M_x, M_y, M_z) = A u, with
//   row 0: 1,  row 1: y_i,  row 2: -x_i,  row 3: s_i k_yaw
// (M = r_i x (0, 0, u_i) = (y_i u_i, -x_i u_i, 0) plus the reaction torque).
struct Rotors {
  int n;             // 4, 6 or 8
  double A[4][8];    // wrench = A u
  double Ap[8][4];   // Moore-Penrose pseudo-inverse A^T (A A^T)^-1
};

inline double rotor_start_angle_deg(int n) { return n == 4 ? 45.0 : (n == 6 ? 30.0 : 22.5); }

// 4x4 inverse by Gauss-Jordan elimination with partial pivoting (FP64).
inline bool invert4(const double in[4][4], double out[4][4]) {
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = j < 4 ? in[i][j] : (j - 4 == i ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (std::fabs(a[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < 8; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
    double d = a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int j = 0; j < 8; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) out[i][j] = a[i][j + 4];
  return true;
}

inline Rotors make_rotors(int n, double arm, double k_yaw) {
  Rotors r{};
  r.n = n;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double beta = (rotor_start_angle_deg(n) + 360.0 * i / n) * pi / 180.0;
    double x = arm * std::cos(beta), y = arm * std::sin(beta);
    double spin = (i % 2 == 0) ? 1.0 : -1.0;
    r.A[0][i] = 1.0;
    r.A[1][i] = y;
    r.A[2][i] = -x;
    r.A[3][i] = spin * k_yaw;
  }
  double AAt[4][4], inv[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += r.A[i][k] * r.A[j][k];
      AAt[i][j] = s;
    }
  invert4(AAt, inv);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int i = 0; i < 4; ++i) s += r.A[i][k] * inv[i][j];
      r.Ap[k][j] = s;
    }
  return r;
}

// Rotor allocation, per-motor clamp and first-order motor lag (one substep):
//   u_cmd = clamp(A^+ (f, M), 0, u_max) per motor,
//   u <- u + alpha (u_cmd - u),  alpha = 1 - exp(-dt_sub / tau)
// (exact zero-order-hold discretisation of tau u' = u_cmd - u; tau = 0 gives
// alpha = 1), then the realised wrench A u, rotor yaw torque included.
template <class T>
Wrench<T> allocate(const Rotors& rot, const Wrench<T>& cmd, T u[8], double u_max, double alpha) {
  T w4[4] = {cmd.f, cmd.M.x, cmd.M.y, cmd.M.z};
  for (int i = 0; i < rot.n; ++i) {
    T uc = T(0);
    for (int j = 0; j < 4; ++j) uc = uc + T(rot.Ap[i][j]) * w4[j];
    uc = clamp(uc, T(0), T(u_max));
    u[i] = u[i] + T(alpha) * (uc - u[i]);
  }
  T out[4];
  for (int j = 0; j < 4; ++j) {
    T s = T(0);
    for (int i = 0; i < rot.n; ++i) s = s + T(rot.A[j][i]) * u[i];
    out[j] = s;
  }
  return Wrench<T>{out[0], Vec3<T>{out[1], out[2], out[3]}};
}

// --------------------------------------------------------------- dynamics --
// Rigid-body 6-DoF dynamics with the wrench held fixed over the substep
// (Sec. I: the robot is a rigid body under thrust and torque):
//   p' = v
//   v' = (f / m) R(q) e_3 - (c_d / m) v + g
//   q' = 1/2 q (x) (0, Omega)
//   Omega' = J^-1 (M - Omega x J Omega)
template <class T> struct Deriv { Vec3<T> dp, dv; Quat<T> dq; Vec3<T> dw; };

template <class T>
Deriv<T> dynamics(const State<T>& s, const Wrench<T>& W, const Body<T>& body, double drag) {
  Deriv<T> d;
  d.dp = s.v;
  d.dv = scale(W.f / body.m, body_z_axis(s.q)) - scale(T(drag) / body.m, s.v) +
         Vec3<T>{T(0), T(0), T(-kGravity)};
  Quat<T> wq = {T(0), s.w.x, s.w.y, s.w.z};
  Quat<T> qw = quat_mul(s.q, wq);
  d.dq = {T(0.5) * qw.w, T(0.5) * qw.x, T(0.5) * qw.y, T(0.5) * qw.z};
  Vec3<T> JW = diag_mul(body.J, s.w);
  Vec3<T> rhs = W.M - cross(s.w, JW);
  d.dw = {rhs.x / body.J.x, rhs.y / body.J.y, rhs.z / body.J.z};
  return d;
}

template <class T> State<T> add_scaled(const State<T>& s, T h, const Deriv<T>& d) {
  State<T> r;
  r.p = s.p + scale(h, d.dp);
  r.v = s.v + scale(h, d.dv);
  r.q = {s.q.w + h * d.dq.w, s.q.x + h * d.dq.x, s.q.y + h * d.dq.y, s.q.z + h * d.dq.z};
  r.w = s.w + scale(h, d.dw);
  return r;
}

// Semi-implicit (symplectic) Euler: velocities first, then positions and
// attitude from the updated velocities; q renormalised afterwards.
template <class T>
State<T> step_sie(const State<T>& s, const Wrench<T>& W, const Body<T>& body, double drag, T h) {
  Deriv<T> d = dynamics(s, W, body, drag);
  State<T> r;
  r.v = s.v + scale(h, d.dv);
  r.w = s.w + scale(h, d.dw);
  r.p = s.p + scale(h, r.v);
  Quat<T> wq = {T(0), r.w.x, r.w.y, r.w.z};
  Quat<T> qw = quat_mul(s.q, wq);
  T hh = T(0.5) * h;
  r.q = quat_normalize(Quat<T>{s.q.w + hh * qw.w, s.q.x + hh * qw.x, s.q.y + hh * qw.y, s.q.z + hh * qw.z});
  return r;
}

// Classic four-stage Runge-Kutta on (p, v, q, Omega) with the wrench held
// fixed over the stages; q renormalised after the step.
template <class T>
State<T> step_rk4(const State<T>& s, const Wrench<T>& W, const Body<T>& body, double drag, T h) {
  T half = T(0.5) * h;
  Deriv<T> k1 = dynamics(s, W, body, drag);
  Deriv<T> k2 = dynamics(add_scaled(s, half, k1), W, body, drag);
  Deriv<T> k3 = dynamics(add_scaled(s, half, k2), W, body, drag);
  Deriv<T> k4 = dynamics(add_scaled(s, h, k3), W, body, drag);
  T c = h / T(6);
  Deriv<T> sum;
  sum.dp = k1.dp + scale(T(2), k2.dp) + scale(T(2), k3.dp) + k4.dp;
  sum.dv = k1.dv + scale(T(2), k2.dv) + scale(T(2), k3.dv) + k4.dv;
  sum.dw = k1.dw + scale(T(2), k2.dw) + scale(T(2), k3.dw) + k4.dw;
  sum.dq = {k1.dq.w + T(2) * k2.dq.w + T(2) * k3.dq.w + k4.dq.w,
            k1.dq.x + T(2) * k2.dq.x + T(2) * k3.dq.x + k4.dq.x,
            k1.dq.y + T(2) * k2.dq.y + T(2) * k3.dq.y + k4.dq.y,
            k1.dq.z + T(2) * k2.dq.z + T(2) * k3.dq.z + k4.dq.z};
  State<T> r = add_scaled(s, c, sum);
  r.q = quat_normalize(r.q);
  return r;
}

// -------------------------------------------------------------- collision --
// Sphere (radius r, centred at the vehicle's centre of mass) versus oriented
// box (centre c, half-extents h, orientation q_b): with d = R(q_b)^T (p - c)
// the sphere centre in the box frame, the closest box point is
// clamp(d, -h, h) and the two touch or overlap iff |d - clamp(d, -h, h)|^2
// <= r^2. This is the collision the paper delegates to the physics engine
// (Sec. I) against the static obstacles of Sec. V. q_b is a unit quaternion.
template <class T>
bool sphere_hits_box(Vec3<T> p, T r, Vec3<T> c, Vec3<T> h, Quat<T> qb) {
  Mat3<T> Rb = unit_quat_to_rot(qb);
  Vec3<T> d = matvec(transpose(Rb), p - c);
  Vec3<T> e = {d.x - clamp(d.x, -h.x, h.x), d.y - clamp(d.y, -h.y, h.y), d.z - clamp(d.z, -h.z, h.z)};
  return !(r * r < dot(e, e));
}

// ------------------------------------------------------------ depth camera --
// Depth image of a pinhole camera against the oriented boxes of one
// environment (the paper renders depth through Isaac Gym's camera sensors,
// Sec. III, and names kernel-based ray casting as its next step, Sec. VII).
// Reading: the camera sits at p + R o_b (o_b its offset in the body frame) and
// looks along body +x with body +z up; pixel (row r, column c) of a W x H
// image with horizontal field of view hfov has the camera-frame ray
//   d = (1, -(c + 0.5 - W/2) / f, -(r + 0.5 - H/2) / f),  f = (W/2) / tan(hfov/2)
// (x forward, y left, z up); the depth of the pixel is the smallest t >= 0
// with o + t R d inside some box, which is the distance along the optical
// axis because d has unit forward component; max_range when nothing is hit
// closer. A ray enters the box {|x_i| <= h_i} (box frame) by the slab method:
// t_in = max_i min(t_i-, t_i+), t_out = min_i max(t_i-, t_i+) with
// t_i-+ = (-+h_i - o_i) / d_i, and hits it iff t_out >= max(t_in, 0).
//
// The work splits into a part per (camera, box) pair, which does not depend on
// the pixel (the box's rotation R_b^T and the camera origin in the box frame),
// and the part per (pixel, box) pair (the ray direction in the box frame and
// the slab intervals). ray_box_depth is the two in sequence.
template <class T> struct BoxInCamera {
  Mat3<T> Rt;   // R_b^T: world -> box frame
  Vec3<T> ob;   // camera origin in the box frame
};

template <class T> BoxInCamera<T> box_in_camera(Vec3<T> o, Vec3<T> c, Quat<T> qb) {
  BoxInCamera<T> bc;
  bc.Rt = transpose(unit_quat_to_rot(qb));
  bc.ob = matvec(bc.Rt, o - c);
  return bc;
}

template <class T> T ray_slab_depth(const BoxInCamera<T>& bc, Vec3<T> d, Vec3<T> h, T max_range) {
  Vec3<T> db = matvec(bc.Rt, d);
  T oi[3] = {bc.ob.x, bc.ob.y, bc.ob.z}, di[3] = {db.x, db.y, db.z}, hi[3] = {h.x, h.y, h.z};
  T t_in = T(-1e300), t_out = T(1e300);
  for (int i = 0; i < 3; ++i) {
    if (di[i] == T(0)) {
      if (oi[i] < -hi[i] || hi[i] < oi[i]) return max_range;  // parallel to the slab and outside it
      continue;
    }
    T t1 = (-hi[i] - oi[i]) / di[i], t2 = (hi[i] - oi[i]) / di[i];
    T lo = t1 < t2 ? t1 : t2, up = t1 < t2 ? t2 : t1;
    if (t_in < lo) t_in = lo;
    if (up < t_out) t_out = up;
  }
  T t0 = t_in < T(0) ? T(0) : t_in;
  if (t_out < t0) return max_range;
  return t0 < max_range ? t0 : max_range;
}

template <class T>
T ray_box_depth(Vec3<T> o, Vec3<T> d, Vec3<T> c, Vec3<T> h, Quat<T> qb, T max_range) {
  return ray_slab_depth(box_in_camera(o, c, qb), d, h, max_range);
}

}  // namespace orc
