// adjoint.cu — differentiable rollout: recorded forward + hand-written adjoint.
//
// Objective (per environment i, over a recorded rollout of H steps):
//   L_i = sum_{t=1..H} ( w_pos |p_t - p_goal,i|^2 + w_omega |Omega_t|^2 ),
// with x_t the state after step t. Gradients are taken with respect to the
// initial state x_0 (13 numbers per environment) and the 12 diagonal
// controller gains (k_x, k_v, k_R, k_Omega), shared by the fleet.
//
// Gradients also go to each environment's four command targets.
//
// The differentiated step is the controller of the environment's command mode
// (position tracking, Sec. I after Lee et al. 2011; body velocity, Eqs. 6-9;
// attitude and thrust, Eqs. 1-2; or a direct wrench) with the attitude law
// of Sec. IV-A (Eqs. 3-5), rotor allocation with per-motor clamp (subgradient
// 0 on a clamped motor) and first-order lag, and the semi-implicit Euler
// update with quaternion renormalisation. Reverse mode is written out by hand, operation by
// operation in reverse order; the comments name the forward line each block
// inverts.
//
// Memory: the forward kernel stores a checkpoint (state + motors) every K
// steps. The backward pass needs every step's start state again. When a tape
// of the whole horizon fits (AdjointBuffers::full_tape), one launch with a
// thread per (vehicle, segment) recomputes every segment's step-start states
// from its checkpoint into the tape at once, and the reverse sweep then reads
// them; otherwise the sweep walks the segments from the last to the first and
// recomputes each segment's states into a one-segment tape itself. Either way
// the sweep recomputes each step's intermediates in registers before
// back-propagating through it. Per-vehicle gain gradients are summed over the
// fleet by a deterministic two-level reduction (fixed block order, fixed tree
// order).
#include <cstdint>
#include <cuda_runtime.h>

#include "adjoint_internal.h"
#include "fleet_device.cuh"

namespace agk {
namespace {

// ----------------------------------------------------------------- forward --
template <int NROT> struct Xs {  // differentiable state of one vehicle
  V3 p, v;
  Q4 q;
  V3 w;
  float u[NROT];
};

// Command of one environment over a recorded rollout: its mode, its four
// targets and the sines and cosines of its angle targets, taken once.
//   position: (c0, s0) = (cos, sin) psi_d
//   attitude: (c0, s0) = (cos, sin) phi_d, (c1, s1) = (cos, sin) theta_d
struct Cmd {
  float t[4];
  float c0, s0, c1, s1;
};

// Intermediates of one forward step, kept for its backward pass.
template <int NROT> struct Step {
  float R[3][3];
  V3 Rd[3];          // columns b1d, b2d, b3d of R_d
  V3 eR, eW;
  float f;           // commanded collective thrust
  float rate;        // commanded yaw rate (velocity, attitude): R_d Omega_d = rate e_3
  // position
  V3 a, c, b1c;      // a is also the vehicle-frame acceleration of the velocity mode
  float ian, icn;    // 1/|a| (0 when |a| <= 1e-9: b3d = e3), 1/|c|
  bool turned;       // heading fallback (b1c turned by 90 degrees) taken
  // current yaw and tilt (velocity, attitude)
  float cps, sps, ir;  // (cos, sin) psi = (R00, R10) * ir; ir = 0 when R00 = R10 = 0
  V3 B[3];             // columns of R_y(theta_d) R_x(phi_d)
  V3 vV;               // velocity in the yaw frame
  float irxz, ianv;    // 1/|(a_x, a_z)|, 1/|a| (both 0 when a_x = a_z = 0)
  // allocation and integration
  float pre[NROT];   // A^+ (f, M) before the clamp
  bool pass[NROT];   // 0 < pre < u_max: the clamp passes the gradient
  float uc[NROT];    // clamped command
  Wrench4 M;         // commanded (f, M)
  Wrench4 W;         // realised wrench
  V3 vn, wn, pn;
  Q4 qt, qn;
  float iqtn;        // 1/|q_t|
};

struct Gains { V3 kx, kv, kR, kW; };

__device__ __forceinline__ Gains gains_of(const StepParams& P) {
  return {{P.kx[0], P.kx[1], P.kx[2]}, {P.kv[0], P.kv[1], P.kv[2]}, {P.kR[0], P.kR[1], P.kR[2]},
          {P.kW[0], P.kW[1], P.kW[2]}};
}

// One recorded step: the controller of mode MODE -> allocation/clamp/lag ->
// SIE. x must hold a unit quaternion.
//   position (Sec. I, Lee 2011): a = -k_x (p - p_d) - k_v v + g e3, f = m a.b3,
//     b3d = a/|a|, b2d = (b3d x b1c)/|.|, b1d = b2d x b3d, Omega_d = 0
//   velocity (Eqs. 6-9): v^V = R_psi^T v, a = k_v (v_d - v^V) + g e3,
//     f = m a.(R_psi^T b3), R_y(theta_d) R_x(phi_d) e3 = a/|a|
//   attitude (Eqs. 1-2): phi_d, theta_d, psi_dot_d, f given
//   velocity and attitude: R_d = R_psi R_y(theta_d) R_x(phi_d) with psi the
//     current yaw, and R_d Omega_d (Eq. 2) = psi_dot_d e3
//   Eqs. 3-5: e_R = 1/2 vee(R_d^T R - R^T R_d), e_W = W - R^T R_d Omega_d,
//     M = -k_R e_R - k_W e_W + W x J W
//   wrench: (f, M) = the targets
template <int NROT, int MODE>
__device__ __forceinline__ void forward_step(const Xs<NROT>& x, const Cmd& cm, const Body& b, const Gains& g,
                                             const StepParams& P, Step<NROT>& S, Xs<NROT>& xn) {
  constexpr int T = NROT == 4 ? 0 : (NROT == 6 ? 1 : 2);
  rotation(x.q, S.R);
  const V3 b3 = {S.R[0][2], S.R[1][2], S.R[2][2]};
  const V3 JW = {b.jx * x.w.x, b.jy * x.w.y, b.jz * x.w.z};
  const V3 gyro = cross(x.w, JW);
  if (MODE == kModeWrench) {
    S.M = {cm.t[0], cm.t[1], cm.t[2], cm.t[3]};
  } else {
    if (MODE == kModePosition) {
      S.a = {-g.kx.x * (x.p.x - cm.t[0]) - g.kv.x * x.v.x, -g.kx.y * (x.p.y - cm.t[1]) - g.kv.y * x.v.y,
             -g.kx.z * (x.p.z - cm.t[2]) - g.kv.z * x.v.z + kGravity};
      S.f = b.m * dot(S.a, b3);
      const float a2 = dot(S.a, S.a);
      S.ian = a2 > 1e-18f ? rsqrt_ftz(a2) : 0.f;
      const V3 b3d = S.ian > 0.f ? S.ian * S.a : V3{0.f, 0.f, 1.f};
      S.b1c = {cm.c0, cm.s0, 0.f};
      S.c = cross(b3d, S.b1c);
      float c2 = dot(S.c, S.c);
      S.turned = !(c2 > 1e-18f);
      if (S.turned) {  // commanded thrust along the heading: use the heading turned by 90 degrees
        S.b1c = {-cm.s0, cm.c0, 0.f};
        S.c = cross(b3d, S.b1c);
        c2 = dot(S.c, S.c);  // near 1
      }
      S.icn = rsqrt_ftz(c2);
      const V3 b2d = S.icn * S.c;
      S.Rd[0] = cross(b2d, b3d);
      S.Rd[1] = b2d;
      S.Rd[2] = b3d;
      S.rate = 0.f;
    } else {
      const float rho2 = S.R[0][0] * S.R[0][0] + S.R[1][0] * S.R[1][0];
      S.ir = rho2 >= kMinNormal ? rsqrt_ftz(rho2) : 0.f;
      S.cps = S.ir > 0.f ? S.R[0][0] * S.ir : 1.f;
      S.sps = S.ir > 0.f ? S.R[1][0] * S.ir : 0.f;
      float cphi, sphi, cth, sth;
      if (MODE == kModeBodyVel) {
        S.vV = {S.cps * x.v.x + S.sps * x.v.y, -S.sps * x.v.x + S.cps * x.v.y, x.v.z};
        S.a = {g.kv.x * (cm.t[0] - S.vV.x), g.kv.y * (cm.t[1] - S.vV.y), g.kv.z * (cm.t[2] - S.vV.z) + kGravity};
        const V3 b3V = {S.cps * b3.x + S.sps * b3.y, -S.sps * b3.x + S.cps * b3.y, b3.z};
        S.f = b.m * dot(S.a, b3V);
        const float rxz2 = S.a.x * S.a.x + S.a.z * S.a.z;
        const float an2 = rxz2 + S.a.y * S.a.y;
        S.irxz = 0.f;
        S.ianv = 0.f;
        cth = 1.f; sth = 0.f; cphi = 1.f; sphi = 0.f;
        if (rxz2 >= kMinNormal) {
          S.irxz = rsqrt_ftz(rxz2);
          S.ianv = rsqrt_ftz(an2);
          cth = S.a.z * S.irxz;
          sth = S.a.x * S.irxz;
          cphi = rxz2 * S.irxz * S.ianv;
          sphi = -S.a.y * S.ianv;
        } else if (an2 > 0.f) {  // a along +-y: phi_d = atan2(-a_y, 0), theta_d = atan2(0, 0) = 0
          cphi = 0.f;
          sphi = S.a.y > 0.f ? -1.f : 1.f;
        }
        S.rate = cm.t[3];
      } else {
        cphi = cm.c0; sphi = cm.s0; cth = cm.c1; sth = cm.s1;
        S.rate = cm.t[2];
        S.f = cm.t[3];
      }
      S.B[0] = {cth, 0.f, -sth};
      S.B[1] = {sth * sphi, cphi, cth * sphi};
      S.B[2] = {sth * cphi, -sphi, cth * cphi};
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S.Rd[j] = {S.cps * S.B[j].x - S.sps * S.B[j].y, S.sps * S.B[j].x + S.cps * S.B[j].y, S.B[j].z};
    }
    // E = R_d^T R: E_ij = col_i(R_d) . col_j(R)
    auto col = [&](int j) { return V3{S.R[0][j], S.R[1][j], S.R[2][j]}; };
    S.eR = {0.5f * (dot(S.Rd[2], col(1)) - dot(S.Rd[1], col(2))),
            0.5f * (dot(S.Rd[0], col(2)) - dot(S.Rd[2], col(0))),
            0.5f * (dot(S.Rd[1], col(0)) - dot(S.Rd[0], col(1)))};
    S.eW = {x.w.x - S.rate * S.R[2][0], x.w.y - S.rate * S.R[2][1], x.w.z - S.rate * S.R[2][2]};
    S.M = {S.f, -g.kR.x * S.eR.x - g.kW.x * S.eW.x + gyro.x, -g.kR.y * S.eR.y - g.kW.y * S.eW.y + gyro.y,
           -g.kR.z * S.eR.z - g.kW.z * S.eW.z + gyro.z};
  }
  S.W = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < NROT; ++i) {
    S.pre[i] = P.Ap[T][i][0] * S.M.f + P.Ap[T][i][1] * S.M.mx + P.Ap[T][i][2] * S.M.my + P.Ap[T][i][3] * S.M.mz;
    S.pass[i] = S.pre[i] > 0.f && S.pre[i] < P.u_max;
    S.uc[i] = fminf(fmaxf(S.pre[i], 0.f), P.u_max);
    xn.u[i] = x.u[i] + P.alpha * (S.uc[i] - x.u[i]);
    S.W.f += P.A[T][0][i] * xn.u[i];
    S.W.mx += P.A[T][1][i] * xn.u[i];
    S.W.my += P.A[T][2][i] * xn.u[i];
    S.W.mz += P.A[T][3][i] * xn.u[i];
  }
  const float h = P.h;
  const float fm = S.W.f * b.inv_m, dm = P.drag * b.inv_m;
  S.vn = {x.v.x + h * (fm * b3.x - dm * x.v.x), x.v.y + h * (fm * b3.y - dm * x.v.y),
          x.v.z + h * (fm * b3.z - dm * x.v.z - kGravity)};
  S.wn = {x.w.x + h * b.ijx * (S.W.mx - gyro.x), x.w.y + h * b.ijy * (S.W.my - gyro.y),
          x.w.z + h * b.ijz * (S.W.mz - gyro.z)};
  S.pn = x.p + h * S.vn;
  const float hh = 0.5f * h;
  const Q4& q = x.q;
  const V3& w = S.wn;
  S.qt = {q.w - hh * (q.x * w.x + q.y * w.y + q.z * w.z), q.x + hh * (q.w * w.x + q.y * w.z - q.z * w.y),
          q.y + hh * (q.w * w.y - q.x * w.z + q.z * w.x), q.z + hh * (q.w * w.z + q.x * w.y - q.y * w.x)};
  S.iqtn = rsqrt_ftz(S.qt.w * S.qt.w + S.qt.x * S.qt.x + S.qt.y * S.qt.y + S.qt.z * S.qt.z);
  const float iq = S.iqtn;
  S.qn = {S.qt.w * iq, S.qt.x * iq, S.qt.y * iq, S.qt.z * iq};
  xn.p = S.pn;
  xn.v = S.vn;
  xn.w = S.wn;
  xn.q = S.qn;
}

// ---------------------------------------------------------------- backward --
template <int NROT> struct Adj {  // adjoint of the state after a step
  V3 p, v;
  Q4 q;
  V3 w;
  float u[NROT];
};

struct GainAdj { V3 kx, kv, kR, kW; };

// d(a x b): a_bar += b x y_bar, b_bar += y_bar x a
__device__ __forceinline__ void cross_bwd(V3 a, V3 b, V3 ybar, V3& abar, V3& bbar) {
  abar = abar + cross(b, ybar);
  bbar = bbar + cross(ybar, a);
}

// y = x / |x| (1 / |x| = in): x_bar += in (y_bar - y (y . y_bar))
__device__ __forceinline__ V3 normalize_bwd(V3 y, float in, V3 ybar) {
  const float d = dot(y, ybar);
  return in * (ybar - d * y);
}

// Reverse of forward_step. On entry lam is the adjoint of (x_{t+1}, u_{t+1})
// including this step's loss term; on exit it is the adjoint of (x_t, u_t).
// Gain adjoints accumulate into gb, target adjoints into tb.
template <int NROT, int MODE>
__device__ __forceinline__ void backward_step(const Xs<NROT>& x, const Cmd& cm, const Body& b, const Gains& g,
                                              const StepParams& P, const Step<NROT>& S, Adj<NROT>& lam, GainAdj& gb,
                                              float (&tb)[4]) {
  constexpr int T = NROT == 4 ? 0 : (NROT == 6 ? 1 : 2);
  const float h = P.h, hh = 0.5f * h;
  const Q4& q = x.q;
  // q_n = q_t / |q_t|
  Q4 qtb;
  {
    const float d = S.qn.w * lam.q.w + S.qn.x * lam.q.x + S.qn.y * lam.q.y + S.qn.z * lam.q.z;
    const float iq = S.iqtn;
    qtb = {iq * (lam.q.w - d * S.qn.w), iq * (lam.q.x - d * S.qn.x), iq * (lam.q.y - d * S.qn.y),
           iq * (lam.q.z - d * S.qn.z)};
  }
  // q_t = q + hh q (x) (0, w_n): linear in q and in w_n
  const V3& w = S.wn;
  Q4 qb = {qtb.w + hh * (qtb.x * w.x + qtb.y * w.y + qtb.z * w.z),
           qtb.x + hh * (-qtb.w * w.x + qtb.y * (-w.z) + qtb.z * w.y),
           qtb.y + hh * (-qtb.w * w.y + qtb.x * w.z - qtb.z * w.x),
           qtb.z + hh * (-qtb.w * w.z - qtb.x * w.y + qtb.y * w.x)};
  V3 wnb = lam.w;
  wnb.x += hh * (-q.x * qtb.w + q.w * qtb.x + q.z * qtb.y - q.y * qtb.z);
  wnb.y += hh * (-q.y * qtb.w - q.z * qtb.x + q.w * qtb.y + q.x * qtb.z);
  wnb.z += hh * (-q.z * qtb.w + q.y * qtb.x - q.x * qtb.y + q.w * qtb.z);
  // p_n = p + h v_n
  V3 pb = lam.p;
  V3 vnb = lam.v + h * lam.p;
  // v_n = v + h (W.f/m b3 - (c/m) v + g)
  const float dm = P.drag * b.inv_m;
  V3 vb = (1.f - h * dm) * vnb;
  const V3 b3 = {S.R[0][2], S.R[1][2], S.R[2][2]};
  Wrench4 Wb;
  Wb.f = h * b.inv_m * dot(b3, vnb);
  V3 Rcb[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, (h * S.W.f * b.inv_m) * vnb};  // adjoints of the columns of R
  // w_n = w + h J^-1 (W.M - gyro(w)), gyro(w) = w x (J w)
  const V3 JW = {b.jx * x.w.x, b.jy * x.w.y, b.jz * x.w.z};
  V3 wb = wnb;
  const V3 jinv_wnb = {h * b.ijx * wnb.x, h * b.ijy * wnb.y, h * b.ijz * wnb.z};
  Wb.mx = jinv_wnb.x;
  Wb.my = jinv_wnb.y;
  Wb.mz = jinv_wnb.z;
  V3 gyrob = {-jinv_wnb.x, -jinv_wnb.y, -jinv_wnb.z};
  // u_{t+1} = u + alpha (uc - u), W = A u_{t+1}
  float ub[NROT], ucb[NROT];
#pragma unroll
  for (int i = 0; i < NROT; ++i) {
    const float un_b = lam.u[i] + P.A[T][0][i] * Wb.f + P.A[T][1][i] * Wb.mx + P.A[T][2][i] * Wb.my +
                       P.A[T][3][i] * Wb.mz;
    ub[i] = (1.f - P.alpha) * un_b;
    ucb[i] = S.pass[i] ? P.alpha * un_b : 0.f;
  }
  // pre = A^+ (f, M)
  Wrench4 Mb = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < NROT; ++i) {
    Mb.f += P.Ap[T][i][0] * ucb[i];
    Mb.mx += P.Ap[T][i][1] * ucb[i];
    Mb.my += P.Ap[T][i][2] * ucb[i];
    Mb.mz += P.Ap[T][i][3] * ucb[i];
  }
  if (MODE == kModeWrench) {
    tb[0] += Mb.f; tb[1] += Mb.mx; tb[2] += Mb.my; tb[3] += Mb.mz;
  } else {
    // M = -k_R e_R - k_W e_W + gyro(w)
    const V3 Mmb = {Mb.mx, Mb.my, Mb.mz};
    gyrob = gyrob + Mmb;
    const V3 eRb = {-g.kR.x * Mb.mx, -g.kR.y * Mb.my, -g.kR.z * Mb.mz};
    const V3 eWb = {-g.kW.x * Mb.mx, -g.kW.y * Mb.my, -g.kW.z * Mb.mz};
    gb.kR = gb.kR - V3{S.eR.x * Mb.mx, S.eR.y * Mb.my, S.eR.z * Mb.mz};
    gb.kW = gb.kW - V3{S.eW.x * Mb.mx, S.eW.y * Mb.my, S.eW.z * Mb.mz};
    // e_W = w - rate (R20, R21, R22)
    wb = wb + eWb;
    Rcb[0].z -= S.rate * eWb.x;
    Rcb[1].z -= S.rate * eWb.y;
    Rcb[2].z -= S.rate * eWb.z;
    const float rateb = -(S.R[2][0] * eWb.x + S.R[2][1] * eWb.y + S.R[2][2] * eWb.z);
    // e_R = 1/2 (E21 - E12, E02 - E20, E10 - E01), E_ij = Rd_i . R_j
    V3 Rdb[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    const V3 Rc[3] = {{S.R[0][0], S.R[1][0], S.R[2][0]}, {S.R[0][1], S.R[1][1], S.R[2][1]}, b3};
    auto Eb = [&](int i, int j, float e) {  // E_ij gets adjoint e
      Rdb[i] = Rdb[i] + e * Rc[j];
      Rcb[j] = Rcb[j] + e * S.Rd[i];
    };
    Eb(2, 1, 0.5f * eRb.x); Eb(1, 2, -0.5f * eRb.x);
    Eb(0, 2, 0.5f * eRb.y); Eb(2, 0, -0.5f * eRb.y);
    Eb(1, 0, 0.5f * eRb.z); Eb(0, 1, -0.5f * eRb.z);
    if (MODE == kModePosition) {
      // f = m a . b3
      V3 ab = (b.m * Mb.f) * b3;
      Rcb[2] = Rcb[2] + (b.m * Mb.f) * S.a;
      // b1d = b2d x b3d
      V3 b2db = Rdb[1], b3db = Rdb[2];
      cross_bwd(S.Rd[1], S.Rd[2], Rdb[0], b2db, b3db);
      // b2d = c / |c|,  c = b3d x b1c
      const V3 cb = normalize_bwd(S.Rd[1], S.icn, b2db);
      V3 b1cb = {0.f, 0.f, 0.f};
      cross_bwd(S.Rd[2], S.b1c, cb, b3db, b1cb);
      // b3d = a / |a| (constant e3 in the degenerate case |a| = 0)
      if (S.ian > 0.f) ab = ab + normalize_bwd(S.Rd[2], S.ian, b3db);
      // a = -k_x (p - p_d) - k_v v + g e3
      const V3 ex = {x.p.x - cm.t[0], x.p.y - cm.t[1], x.p.z - cm.t[2]};
      pb = pb - V3{g.kx.x * ab.x, g.kx.y * ab.y, g.kx.z * ab.z};
      vb = vb - V3{g.kv.x * ab.x, g.kv.y * ab.y, g.kv.z * ab.z};
      gb.kx = gb.kx - V3{ex.x * ab.x, ex.y * ab.y, ex.z * ab.z};
      gb.kv = gb.kv - V3{x.v.x * ab.x, x.v.y * ab.y, x.v.z * ab.z};
      tb[0] += g.kx.x * ab.x;
      tb[1] += g.kx.y * ab.y;
      tb[2] += g.kx.z * ab.z;
      // b1c = (cos psi_d, sin psi_d, 0), or (-sin psi_d, cos psi_d, 0) when turned
      tb[3] += S.turned ? -cm.c0 * b1cb.x - cm.s0 * b1cb.y : -cm.s0 * b1cb.x + cm.c0 * b1cb.y;
    } else {
      // R_d = R_psi B: adjoints of B's columns and of (cos psi, sin psi)
      V3 Bb[3];
      float cpb = 0.f, spb = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Bb[j] = {S.cps * Rdb[j].x + S.sps * Rdb[j].y, -S.sps * Rdb[j].x + S.cps * Rdb[j].y, Rdb[j].z};
        cpb += Rdb[j].x * S.B[j].x + Rdb[j].y * S.B[j].y;
        spb += -Rdb[j].x * S.B[j].y + Rdb[j].y * S.B[j].x;
      }
      if (MODE == kModeAttThrust) {
        // B = R_y(theta_d) R_x(phi_d): columns (ct, 0, -st), (st sp, cp, ct sp), (st cp, -sp, ct cp)
        const float cp = cm.c0, sp = cm.s0, ct = cm.c1, st = cm.s1;
        const float thb = Bb[0].x * -st + Bb[0].z * -ct + Bb[1].x * (ct * sp) + Bb[1].z * (-st * sp) +
                          Bb[2].x * (ct * cp) + Bb[2].z * (-st * cp);
        const float phb = Bb[1].x * (st * cp) + Bb[1].y * -sp + Bb[1].z * (ct * cp) + Bb[2].x * (-st * sp) +
                          Bb[2].y * -cp + Bb[2].z * (-ct * sp);
        tb[0] += phb;
        tb[1] += thb;
        tb[2] += rateb;
        tb[3] += Mb.f;
      } else {
        // f = m a . b3V, b3V = R_psi^T b3
        const V3 b3V = {S.cps * b3.x + S.sps * b3.y, -S.sps * b3.x + S.cps * b3.y, b3.z};
        V3 ab = (b.m * Mb.f) * b3V;
        const V3 b3Vb = (b.m * Mb.f) * S.a;
        Rcb[2].x += S.cps * b3Vb.x - S.sps * b3Vb.y;
        Rcb[2].y += S.sps * b3Vb.x + S.cps * b3Vb.y;
        Rcb[2].z += b3Vb.z;
        cpb += b3.x * b3Vb.x + b3.y * b3Vb.y;
        spb += b3.y * b3Vb.x - b3.x * b3Vb.y;
        // B from a: B_2 = a/|a|, B_0 = (a_z, 0, -a_x)/|(a_x, a_z)|, B_1 = B_2 x B_0 (constant when a_x = a_z = 0)
        if (S.irxz > 0.f) {
          V3 B2b = Bb[2], B0b = Bb[0];
          cross_bwd(S.B[2], S.B[0], Bb[1], B2b, B0b);
          const V3 wbar = normalize_bwd(S.B[0], S.irxz, B0b);
          ab.z += wbar.x;
          ab.x -= wbar.z;
          ab = ab + normalize_bwd(S.B[2], S.ianv, B2b);
        }
        // a = k_v (v_d - v^V) + g e3
        const V3 vVb = {-g.kv.x * ab.x, -g.kv.y * ab.y, -g.kv.z * ab.z};
        tb[0] += g.kv.x * ab.x;
        tb[1] += g.kv.y * ab.y;
        tb[2] += g.kv.z * ab.z;
        gb.kv = gb.kv + V3{(cm.t[0] - S.vV.x) * ab.x, (cm.t[1] - S.vV.y) * ab.y, (cm.t[2] - S.vV.z) * ab.z};
        // v^V = R_psi^T v
        vb.x += S.cps * vVb.x - S.sps * vVb.y;
        vb.y += S.sps * vVb.x + S.cps * vVb.y;
        vb.z += vVb.z;
        cpb += x.v.x * vVb.x + x.v.y * vVb.y;
        spb += x.v.y * vVb.x - x.v.x * vVb.y;
        tb[3] += rateb;
      }
      // (cos psi, sin psi) = (R00, R10) / |(R00, R10)|
      if (S.ir > 0.f) {
        const float d = S.cps * cpb + S.sps * spb;
        Rcb[0].x += S.ir * (cpb - d * S.cps);
        Rcb[0].y += S.ir * (spb - d * S.sps);
      }
    }
  }
  // gyro = w x (J w): w_bar += (J w) x g_bar + J (g_bar x w)
  {
    V3 jwb = {0.f, 0.f, 0.f};
    cross_bwd(x.w, JW, gyrob, wb, jwb);
    wb = wb + V3{b.jx * jwb.x, b.jy * jwb.y, b.jz * jwb.z};
  }
  // R = R(q), unit-quaternion formula; Rcb[j] is the adjoint of column j
  {
    const float w0 = q.w, x0 = q.x, y0 = q.y, z0 = q.z;
    const float R00 = Rcb[0].x, R10 = Rcb[0].y, R20 = Rcb[0].z;
    const float R01 = Rcb[1].x, R11 = Rcb[1].y, R21 = Rcb[1].z;
    const float R02 = Rcb[2].x, R12 = Rcb[2].y, R22 = Rcb[2].z;
    // R00 = 1-2(y2+z2), R01 = 2(xy-wz), R02 = 2(xz+wy), R10 = 2(xy+wz), R11 = 1-2(x2+z2),
    // R12 = 2(yz-wx), R20 = 2(xz-wy), R21 = 2(yz+wx), R22 = 1-2(x2+y2)
    qb.w += 2.f * (-z0 * R01 + y0 * R02 + z0 * R10 - x0 * R12 - y0 * R20 + x0 * R21);
    qb.x += 2.f * (y0 * R01 + z0 * R02 + y0 * R10 - 2.f * x0 * R11 - w0 * R12 + z0 * R20 + w0 * R21 -
                   2.f * x0 * R22);
    qb.y += 2.f * (-2.f * y0 * R00 + x0 * R01 + w0 * R02 + x0 * R10 + z0 * R12 - w0 * R20 + z0 * R21 -
                   2.f * y0 * R22);
    qb.z += 2.f * (-2.f * z0 * R00 - w0 * R01 + x0 * R02 + w0 * R10 - 2.f * z0 * R11 + y0 * R12 + x0 * R20 +
                   y0 * R21);
  }
  lam.p = pb;
  lam.v = vb;
  lam.q = qb;
  lam.w = wb;
#pragma unroll
  for (int i = 0; i < NROT; ++i) lam.u[i] = ub[i];
}

// ----------------------------------------------------------------- kernels --
template <int NROT>
__device__ __forceinline__ void load_x(const float* st, const float* mot, uint32_t n, uint32_t i, Xs<NROT>& x) {
  x.p = {st[0 * n + i], st[1 * n + i], st[2 * n + i]};
  x.v = {st[3 * n + i], st[4 * n + i], st[5 * n + i]};
  x.q = {st[6 * n + i], st[7 * n + i], st[8 * n + i], st[9 * n + i]};
  x.w = {st[10 * n + i], st[11 * n + i], st[12 * n + i]};
#pragma unroll
  for (int k = 0; k < NROT; ++k) x.u[k] = mot[k * n + i];
}

template <int NROT>
__device__ __forceinline__ void store_x(float* st, float* mot, uint32_t n, uint32_t i, const Xs<NROT>& x) {
  st[0 * n + i] = x.p.x; st[1 * n + i] = x.p.y; st[2 * n + i] = x.p.z;
  st[3 * n + i] = x.v.x; st[4 * n + i] = x.v.y; st[5 * n + i] = x.v.z;
  st[6 * n + i] = x.q.w; st[7 * n + i] = x.q.x; st[8 * n + i] = x.q.y; st[9 * n + i] = x.q.z;
  st[10 * n + i] = x.w.x; st[11 * n + i] = x.w.y; st[12 * n + i] = x.w.z;
#pragma unroll
  for (int k = 0; k < NROT; ++k) mot[k * n + i] = x.u[k];
}

__device__ __forceinline__ Body body_at(const float* bd, uint32_t n, uint32_t i) {
  return make_body(bd[i], bd[n + i], bd[2 * n + i], bd[3 * n + i]);
}

__device__ __forceinline__ int rotors_of(const AdjointBuffers& ab, uint32_t i) {
  return i < ab.n_quad ? 4 : (i < ab.n_quad + ab.n_hexa ? 6 : 8);
}

__device__ __forceinline__ Cmd load_cmd(const AdjointBuffers& ab, uint32_t i, int mode) {
  const uint32_t n = ab.n;
  Cmd cm;
#pragma unroll
  for (int k = 0; k < 4; ++k) cm.t[k] = ab.targets[k * n + i];
  cm.c0 = 1.f; cm.s0 = 0.f; cm.c1 = 1.f; cm.s1 = 0.f;
  if (mode == kModePosition) sincosf(cm.t[3], &cm.s0, &cm.c0);
  if (mode == kModeAttThrust) {
    sincosf(cm.t[0], &cm.s0, &cm.c0);
    sincosf(cm.t[1], &cm.s1, &cm.c1);
  }
  return cm;
}

__device__ __forceinline__ int mode_of(const AdjointBuffers& ab, uint32_t i) {
  const int m = ab.modes[i];
  return m > kModeWrench ? kModeWrench : m;
}

// Forward recording: n_steps steps from the fleet state, checkpoint (state,
// motors) every K steps into ckpt[s][13 + 8][n], loss per env, final state
// written back, saturation flag per env.
template <int NROT, int MODE>
__device__ void record_one(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  const uint32_t n = ab.n;
  Xs<NROT> x;
  load_x(ab.state, ab.motors, n, i, x);
  store_x(ab.ckpt, ab.ckpt + 13 * n, n, i, x);  // checkpoint 0 keeps the raw (possibly non-unit) q_0
  normalize(x.q);
  const Body b = body_at(ab.body, n, i);
  const Gains g = gains_of(P);
  const Cmd cm = load_cmd(ab, i, MODE);
  const V3 goal = {ab.p_goal[i], ab.p_goal[n + i], ab.p_goal[2 * n + i]};
  float loss = 0.f;
  bool saturated = false;
  for (int t = 0; t < ab.n_steps; ++t) {
    if (t > 0 && t % ab.K == 0)
      store_x(ab.ckpt + (size_t)(t / ab.K) * 21 * n, ab.ckpt + (size_t)(t / ab.K) * 21 * n + 13 * n, n, i, x);
    Step<NROT> S;
    Xs<NROT> xn;
    forward_step<NROT, MODE>(x, cm, b, g, P, S, xn);
#pragma unroll
    for (int k = 0; k < NROT; ++k) saturated |= !S.pass[k];
    x = xn;
    const V3 e = x.p - goal;
    loss += ab.w_pos * dot(e, e) + ab.w_omega * dot(x.w, x.w);
  }
  store_x(ab.state, ab.motors, n, i, x);
  ab.loss[i] = loss;
  ab.saturated[i] = saturated ? 1 : 0;
}

template <int NROT>
__device__ __forceinline__ void record_mode(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  switch (mode_of(ab, i)) {
    case kModePosition: record_one<NROT, kModePosition>(ab, P, i); break;
    case kModeBodyVel: record_one<NROT, kModeBodyVel>(ab, P, i); break;
    case kModeAttThrust: record_one<NROT, kModeAttThrust>(ab, P, i); break;
    default: record_one<NROT, kModeWrench>(ab, P, i); break;
  }
}

// One warp per block: the fleet's warps spread evenly over the SMs (a
// 65,536-vehicle fleet puts 13 or 14 on each of 152 SMs, where 128-thread
// blocks would put 12 on some and 16 on others).
constexpr int kRecordBlock = 32;
__global__ void __launch_bounds__(kRecordBlock) k_record(AdjointBuffers ab, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ab.n) return;
  const int nr = rotors_of(ab, i);
  if (nr == 4) record_mode<4>(ab, P, i);
  else if (nr == 6) record_mode<6>(ab, P, i);
  else record_mode<8>(ab, P, i);
}

// Adjoint state of one vehicle during the reverse sweep.
template <int NROT> struct SweepState {
  Adj<NROT> lam;
  GainAdj gb;
  float tb[4];
};

template <int NROT> __device__ __forceinline__ void sweep_init(SweepState<NROT>& z) {
  z.lam.p = z.lam.v = z.lam.w = {0.f, 0.f, 0.f};
  z.lam.q = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < NROT; ++k) z.lam.u[k] = 0.f;
  z.gb.kx = z.gb.kv = z.gb.kR = z.gb.kW = {0.f, 0.f, 0.f};
  z.tb[0] = z.tb[1] = z.tb[2] = z.tb[3] = 0.f;
}

// One step of the reverse sweep from its start state x: recompute the step's
// intermediates, add the step's loss term (it acts on x_{t+1}), back-propagate.
template <int NROT, int MODE>
__device__ __forceinline__ void sweep_step(const AdjointBuffers& ab, const StepParams& P, const Xs<NROT>& x,
                                           const Cmd& cm, const Body& b, const Gains& g, V3 goal, float wgt,
                                           SweepState<NROT>& z) {
  Step<NROT> S;
  Xs<NROT> xn;
  forward_step<NROT, MODE>(x, cm, b, g, P, S, xn);
  const V3 e = xn.p - goal;
  z.lam.p = z.lam.p + (2.f * ab.w_pos * wgt) * e;
  z.lam.w = z.lam.w + (2.f * ab.w_omega * wgt) * xn.w;
  backward_step<NROT, MODE>(x, cm, b, g, P, S, z.lam, z.gb, z.tb);
}

// Writes vehicle i's gradients. The kernel normalised q_0 at load
// (q_hat = q0 / |q0|), so the quaternion adjoint is mapped back through that.
template <int NROT>
__device__ __forceinline__ void sweep_finish(const AdjointBuffers& ab, uint32_t i, SweepState<NROT>& z) {
  const uint32_t n = ab.n;
  Adj<NROT>& lam = z.lam;
  {
    const Q4 q0 = {ab.ckpt[6 * n + i], ab.ckpt[7 * n + i], ab.ckpt[8 * n + i], ab.ckpt[9 * n + i]};
    const float nq = sqrtf(q0.w * q0.w + q0.x * q0.x + q0.y * q0.y + q0.z * q0.z);
    const Q4 qh = {q0.w / nq, q0.x / nq, q0.y / nq, q0.z / nq};
    const float d = qh.w * lam.q.w + qh.x * lam.q.x + qh.y * lam.q.y + qh.z * lam.q.z;
    lam.q = {(lam.q.w - d * qh.w) / nq, (lam.q.x - d * qh.x) / nq, (lam.q.y - d * qh.y) / nq,
             (lam.q.z - d * qh.z) / nq};
  }
  float* gx = ab.grad_x0;
  gx[0 * n + i] = lam.p.x; gx[1 * n + i] = lam.p.y; gx[2 * n + i] = lam.p.z;
  gx[3 * n + i] = lam.v.x; gx[4 * n + i] = lam.v.y; gx[5 * n + i] = lam.v.z;
  gx[6 * n + i] = lam.q.w; gx[7 * n + i] = lam.q.x; gx[8 * n + i] = lam.q.y; gx[9 * n + i] = lam.q.z;
  gx[10 * n + i] = lam.w.x; gx[11 * n + i] = lam.w.y; gx[12 * n + i] = lam.w.z;
  float* gg = ab.grad_gains_env;
  const GainAdj& gb = z.gb;
  const float v12[12] = {gb.kx.x, gb.kx.y, gb.kx.z, gb.kv.x, gb.kv.y, gb.kv.z,
                         gb.kR.x, gb.kR.y, gb.kR.z, gb.kW.x, gb.kW.y, gb.kW.z};
#pragma unroll
  for (int k = 0; k < 12; ++k) gg[k * n + i] = v12[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) ab.grad_targets[k * n + i] = z.tb[k];
}

template <int NROT>
__device__ __forceinline__ float* tape_at(const AdjointBuffers& ab, int t) {
  return ab.tape + (size_t)t * 21 * ab.n;
}

// Reverse sweep of vehicle i. full_tape: every step-start state is already on
// the tape (k_tape); otherwise each segment's states are recomputed here,
// segment by segment, into the one-segment tape.
template <int NROT, int MODE, bool FULL_TAPE>
__device__ void adjoint_one(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  const uint32_t n = ab.n;
  const Body b = body_at(ab.body, n, i);
  const Gains g = gains_of(P);
  const Cmd cm = load_cmd(ab, i, MODE);
  const V3 goal = {ab.p_goal[i], ab.p_goal[n + i], ab.p_goal[2 * n + i]};
  const float wgt = ab.loss_weights ? ab.loss_weights[i] : 1.f;
  SweepState<NROT> z;
  sweep_init(z);
  const int H = ab.n_steps, K = ab.K;
  if (FULL_TAPE) {
    // the next (earlier) tape entry is requested one step ahead
    Xs<NROT> x, x_prev;
    load_x(tape_at<NROT>(ab, H - 1), tape_at<NROT>(ab, H - 1) + 13 * n, n, i, x_prev);
    for (int t = H - 1; t >= 0; --t) {
      x = x_prev;
      if (t > 0) load_x(tape_at<NROT>(ab, t - 1), tape_at<NROT>(ab, t - 1) + 13 * n, n, i, x_prev);
      sweep_step<NROT, MODE>(ab, P, x, cm, b, g, goal, wgt, z);
    }
    sweep_finish(ab, i, z);
    return;
  }
  const int n_seg = (H + K - 1) / K;
  for (int seg = n_seg - 1; seg >= 0; --seg) {
    const int t0 = seg * K;
    const int len = H - t0 < K ? H - t0 : K;
    Xs<NROT> x;
    load_x(ab.ckpt + (size_t)seg * 21 * n, ab.ckpt + (size_t)seg * 21 * n + 13 * n, n, i, x);
    if (seg == 0) normalize(x.q);
    // recompute the segment's step-start states into the tape
    for (int t = 0; t < len; ++t) {
      store_x(tape_at<NROT>(ab, t), tape_at<NROT>(ab, t) + 13 * n, n, i, x);
      if (t + 1 < len) {
        Step<NROT> S;
        Xs<NROT> xn;
        forward_step<NROT, MODE>(x, cm, b, g, P, S, xn);
        x = xn;
      }
    }
    // reverse sweep; the next (earlier) tape entry is requested one step ahead
    Xs<NROT> x_prev;
    load_x(tape_at<NROT>(ab, len - 1), tape_at<NROT>(ab, len - 1) + 13 * n, n, i, x_prev);
    for (int t = len - 1; t >= 0; --t) {
      x = x_prev;
      if (t > 0) load_x(tape_at<NROT>(ab, t - 1), tape_at<NROT>(ab, t - 1) + 13 * n, n, i, x_prev);
      sweep_step<NROT, MODE>(ab, P, x, cm, b, g, goal, wgt, z);
    }
  }
  sweep_finish(ab, i, z);
}

// Step-start states of one segment of vehicle i, recomputed from its
// checkpoint into the whole-horizon tape (tape step t0 + t, t < len).
template <int NROT, int MODE>
__device__ void tape_one(const AdjointBuffers& ab, const StepParams& P, uint32_t i, int seg) {
  const uint32_t n = ab.n;
  const int t0 = seg * ab.K;
  const int len = ab.n_steps - t0 < ab.K ? ab.n_steps - t0 : ab.K;
  const Body b = body_at(ab.body, n, i);
  const Gains g = gains_of(P);
  const Cmd cm = load_cmd(ab, i, MODE);
  Xs<NROT> x;
  load_x(ab.ckpt + (size_t)seg * 21 * n, ab.ckpt + (size_t)seg * 21 * n + 13 * n, n, i, x);
  if (seg == 0) normalize(x.q);
  for (int t = 0; t < len; ++t) {
    store_x(tape_at<NROT>(ab, t0 + t), tape_at<NROT>(ab, t0 + t) + 13 * n, n, i, x);
    if (t + 1 < len) {
      Step<NROT> S;
      Xs<NROT> xn;
      forward_step<NROT, MODE>(x, cm, b, g, P, S, xn);
      x = xn;
    }
  }
}

template <int NROT>
__device__ __forceinline__ void tape_mode(const AdjointBuffers& ab, const StepParams& P, uint32_t i, int seg) {
  switch (mode_of(ab, i)) {
    case kModePosition: tape_one<NROT, kModePosition>(ab, P, i, seg); break;
    case kModeBodyVel: tape_one<NROT, kModeBodyVel>(ab, P, i, seg); break;
    case kModeAttThrust: tape_one<NROT, kModeAttThrust>(ab, P, i, seg); break;
    default: tape_one<NROT, kModeWrench>(ab, P, i, seg); break;
  }
}

// One thread per (vehicle, segment): thread j handles vehicle j % n of
// segment j / n, so a warp's loads and stores stay coalesced.
constexpr int kTapeBlock = 128;
__global__ void __launch_bounds__(kTapeBlock) k_tape(AdjointBuffers ab, StepParams P, int n_seg) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (uint64_t)ab.n * n_seg) return;
  const uint32_t i = (uint32_t)(j % ab.n);
  const int seg = (int)(j / ab.n);
  const int nr = rotors_of(ab, i);
  if (nr == 4) tape_mode<4>(ab, P, i, seg);
  else if (nr == 6) tape_mode<6>(ab, P, i, seg);
  else tape_mode<8>(ab, P, i, seg);
}

template <int NROT, bool FULL_TAPE>
__device__ __forceinline__ void adjoint_mode(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  switch (mode_of(ab, i)) {
    case kModePosition: adjoint_one<NROT, kModePosition, FULL_TAPE>(ab, P, i); break;
    case kModeBodyVel: adjoint_one<NROT, kModeBodyVel, FULL_TAPE>(ab, P, i); break;
    case kModeAttThrust: adjoint_one<NROT, kModeAttThrust, FULL_TAPE>(ab, P, i); break;
    default: adjoint_one<NROT, kModeWrench, FULL_TAPE>(ab, P, i); break;
  }
}

// One warp per block and at most 128 registers. Each SM sub-partition holds a
// quarter of the register file: 128 registers fit four warps per
// sub-partition, 16 per SM, so a 65,536-vehicle fleet (2,048 warps) is
// resident in one wave on 152 SMs, and single-warp blocks spread the warps
// evenly (13 or 14 per SM). The sweep wants about 168 registers, and the cap
// spills about 1.3 KB per thread; at 144 registers (12 warps per SM) the
// fleet needed 1.12 waves, which cost more than the spills do.
constexpr int kAdjointBlock = 32;
template <bool FULL_TAPE>
__global__ void __maxnreg__(128) k_adjoint(AdjointBuffers ab, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ab.n) return;
  const int nr = rotors_of(ab, i);
  if (nr == 4) adjoint_mode<4, FULL_TAPE>(ab, P, i);
  else if (nr == 6) adjoint_mode<6, FULL_TAPE>(ab, P, i);
  else adjoint_mode<8, FULL_TAPE>(ab, P, i);
}

// Deterministic fleet sum of the 12 per-env gain gradients: each of the
// `parts` blocks sums a fixed contiguous range in a fixed tree order into
// partial[k][block]; one block then sums the partials in the same way.
constexpr int kRedThreads = 256;

__device__ __forceinline__ float block_tree_sum(float v, float* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  float r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(const float* per_env, uint32_t n, float* partial,
                                                                int parts) {
  __shared__ float sh[kRedThreads];
  const int k = blockIdx.y;
  const size_t chunk = (n + parts - 1) / parts;
  const size_t lo = chunk * blockIdx.x, hi = lo + chunk < n ? lo + chunk : n;
  float acc = 0.f;
  for (size_t j = lo + threadIdx.x; j < hi; j += kRedThreads) acc += per_env[(size_t)k * n + j];
  const float s = block_tree_sum(acc, sh);
  if (threadIdx.x == 0) partial[k * parts + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const float* partial, int parts, float* out) {
  __shared__ float sh[kRedThreads];
  const int k = blockIdx.x;
  float acc = 0.f;
  for (int j = threadIdx.x; j < parts; j += kRedThreads) acc += partial[k * parts + j];
  const float s = block_tree_sum(acc, sh);
  if (threadIdx.x == 0) out[k] = s;
}

}  // namespace

cudaError_t launch_record(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st) {
  k_record<<<(ab.n + kRecordBlock - 1) / kRecordBlock, kRecordBlock, 0, st>>>(ab, P);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st) {
  cudaError_t e;
  if (ab.full_tape) {
    const int n_seg = (ab.n_steps + ab.K - 1) / ab.K;
    const uint64_t threads = (uint64_t)ab.n * n_seg;
    k_tape<<<(unsigned)((threads + kTapeBlock - 1) / kTapeBlock), kTapeBlock, 0, st>>>(ab, P, n_seg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const unsigned blocks = (ab.n + kAdjointBlock - 1) / kAdjointBlock;
  if (ab.full_tape) k_adjoint<true><<<blocks, kAdjointBlock, 0, st>>>(ab, P);
  else k_adjoint<false><<<blocks, kAdjointBlock, 0, st>>>(ab, P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g1(kReduceParts, 12);
  k_reduce_partial<<<g1, kRedThreads, 0, st>>>(ab.grad_gains_env, ab.n, ab.partial, kReduceParts);
  k_reduce_final<<<12, kRedThreads, 0, st>>>(ab.partial, kReduceParts, ab.grad_gains);
  return cudaGetLastError();
}

}  // namespace agk
