// adjoint.cu — differentiable rollout: recorded forward + hand-written adjoint.
//
// Objective (per environment i, over a recorded rollout of H steps):
//   L_i = sum_{t=1..H} ( w_pos |p_t - p_goal,i|^2 + w_omega |Omega_t|^2 ),
// with x_t the state after step t. Gradients are taken with respect to the
// initial state x_0 (13 numbers per environment) and the 12 diagonal
// controller gains (k_x, k_v, k_R, k_Omega), shared by the fleet.
//
// The differentiated step is the position-tracking controller (Sec. I, after
// Lee et al. 2011) with the attitude law of Sec. IV-A (Eqs. 3-5), rotor
// allocation with per-motor clamp (subgradient 0 on a clamped motor) and
// first-order lag, and the semi-implicit Euler update with quaternion
// renormalisation. Reverse mode is written out by hand, operation by
// operation in reverse order; the comments name the forward line each block
// inverts.
//
// Memory: the forward kernel stores a checkpoint (state + motors) every K
// steps. The adjoint kernel walks the segments from the last to the first:
// it recomputes the segment's K step-start states into a per-vehicle tape,
// then sweeps them in reverse, recomputing each step's intermediates in
// registers before back-propagating through it. Per-vehicle gain gradients
// are summed over the fleet by a deterministic two-level reduction (fixed
// block order, fixed tree order).
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

// Intermediates of one forward step, kept for its backward pass.
template <int NROT> struct Step {
  float R[3][3];
  V3 a, b3d, b1c, c, b2d, b1d, eR;
  float an, cn, f;
  float pre[NROT];   // A^+ (f, M) before the clamp
  bool pass[NROT];   // 0 < pre < u_max: the clamp passes the gradient
  float uc[NROT];    // clamped command
  Wrench4 M;         // commanded (f, M)
  Wrench4 W;         // realised wrench
  V3 vn, wn, pn;
  Q4 qt, qn;
  float qtn;
};

struct Gains { V3 kx, kv, kR, kW; };

__device__ __forceinline__ Gains gains_of(const StepParams& P) {
  return {{P.kx[0], P.kx[1], P.kx[2]}, {P.kv[0], P.kv[1], P.kv[2]}, {P.kR[0], P.kR[1], P.kR[2]},
          {P.kW[0], P.kW[1], P.kW[2]}};
}

// One recorded step: position controller -> allocation/clamp/lag -> SIE.
// x must hold a unit quaternion.
template <int NROT>
__device__ __forceinline__ void forward_step(const Xs<NROT>& x, V3 pd, float cpsi, float spsi, const Body& b,
                                             const Gains& g, const StepParams& P, Step<NROT>& S, Xs<NROT>& xn) {
  constexpr int T = NROT == 4 ? 0 : (NROT == 6 ? 1 : 2);
  rotation(x.q, S.R);
  V3 b3 = {S.R[0][2], S.R[1][2], S.R[2][2]};
  S.a = {-g.kx.x * (x.p.x - pd.x) - g.kv.x * x.v.x, -g.kx.y * (x.p.y - pd.y) - g.kv.y * x.v.y,
         -g.kx.z * (x.p.z - pd.z) - g.kv.z * x.v.z + kGravity};
  S.f = b.m * dot(S.a, b3);
  S.an = sqrtf(dot(S.a, S.a));
  S.b3d = S.an > 1e-9f ? (1.f / S.an) * S.a : V3{0.f, 0.f, 1.f};
  S.b1c = {cpsi, spsi, 0.f};
  S.c = cross(S.b3d, S.b1c);
  S.cn = sqrtf(dot(S.c, S.c));
  if (!(S.cn > 1e-9f)) {  // commanded thrust along the heading: use the heading turned by 90 degrees
    S.b1c = {-spsi, cpsi, 0.f};
    S.c = cross(S.b3d, S.b1c);
    S.cn = sqrtf(dot(S.c, S.c));
  }
  S.b2d = (1.f / S.cn) * S.c;
  S.b1d = cross(S.b2d, S.b3d);
  // E = R_d^T R with R_d = [b1d b2d b3d]: E_ij = col_i(R_d) . col_j(R)
  V3 Rd[3] = {S.b1d, S.b2d, S.b3d};
  auto col = [&](int j) { return V3{S.R[0][j], S.R[1][j], S.R[2][j]}; };
  S.eR = {0.5f * (dot(Rd[2], col(1)) - dot(Rd[1], col(2))), 0.5f * (dot(Rd[0], col(2)) - dot(Rd[2], col(0))),
          0.5f * (dot(Rd[1], col(0)) - dot(Rd[0], col(1)))};
  V3 JW = {b.jx * x.w.x, b.jy * x.w.y, b.jz * x.w.z};
  V3 gyro = cross(x.w, JW);
  S.M = {S.f, -g.kR.x * S.eR.x - g.kW.x * x.w.x + gyro.x, -g.kR.y * S.eR.y - g.kW.y * x.w.y + gyro.y,
         -g.kR.z * S.eR.z - g.kW.z * x.w.z + gyro.z};
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
  S.qtn = sqrtf(S.qt.w * S.qt.w + S.qt.x * S.qt.x + S.qt.y * S.qt.y + S.qt.z * S.qt.z);
  const float iq = 1.f / S.qtn;
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

// y = x / |x| (|x| = n): x_bar += (y_bar - y (y . y_bar)) / n
__device__ __forceinline__ V3 normalize_bwd(V3 y, float n, V3 ybar) {
  const float d = dot(y, ybar);
  return (1.f / n) * (ybar - d * y);
}

// Reverse of forward_step. On entry lam is the adjoint of (x_{t+1}, u_{t+1})
// including this step's loss term; on exit it is the adjoint of (x_t, u_t).
template <int NROT>
__device__ __forceinline__ void backward_step(const Xs<NROT>& x, V3 pd, float cpsi, float spsi, const Body& b,
                                              const Gains& g, const StepParams& P, const Step<NROT>& S,
                                              Adj<NROT>& lam, GainAdj& gb) {
  constexpr int T = NROT == 4 ? 0 : (NROT == 6 ? 1 : 2);
  const float h = P.h, hh = 0.5f * h;
  const Q4& q = x.q;
  // q_n = q_t / |q_t|
  Q4 qtb;
  {
    const float d = S.qn.w * lam.q.w + S.qn.x * lam.q.x + S.qn.y * lam.q.y + S.qn.z * lam.q.z;
    const float iq = 1.f / S.qtn;
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
  V3 b3b = (h * S.W.f * b.inv_m) * vnb;
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
  // M = -k_R e_R - k_W w + gyro(w)
  const V3 Mmb = {Mb.mx, Mb.my, Mb.mz};
  gyrob = gyrob + Mmb;
  V3 eRb = {-g.kR.x * Mb.mx, -g.kR.y * Mb.my, -g.kR.z * Mb.mz};
  wb = wb - V3{g.kW.x * Mb.mx, g.kW.y * Mb.my, g.kW.z * Mb.mz};
  gb.kR = gb.kR - V3{S.eR.x * Mb.mx, S.eR.y * Mb.my, S.eR.z * Mb.mz};
  gb.kW = gb.kW - V3{x.w.x * Mb.mx, x.w.y * Mb.my, x.w.z * Mb.mz};
  // gyro = w x (J w): w_bar += (J w) x g_bar + J (g_bar x w)
  {
    V3 jwb = {0.f, 0.f, 0.f};
    cross_bwd(x.w, JW, gyrob, wb, jwb);
    wb = wb + V3{b.jx * jwb.x, b.jy * jwb.y, b.jz * jwb.z};
  }
  // e_R = 1/2 (E21 - E12, E02 - E20, E10 - E01), E_ij = Rd_i . R_j
  V3 Rdb[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  V3 Rcb[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  const V3 Rd[3] = {S.b1d, S.b2d, S.b3d};
  const V3 Rc[3] = {{S.R[0][0], S.R[1][0], S.R[2][0]}, {S.R[0][1], S.R[1][1], S.R[2][1]}, b3};
  auto Eb = [&](int i, int j, float e) {  // E_ij gets adjoint e
    Rdb[i] = Rdb[i] + e * Rc[j];
    Rcb[j] = Rcb[j] + e * Rd[i];
  };
  Eb(2, 1, 0.5f * eRb.x); Eb(1, 2, -0.5f * eRb.x);
  Eb(0, 2, 0.5f * eRb.y); Eb(2, 0, -0.5f * eRb.y);
  Eb(1, 0, 0.5f * eRb.z); Eb(0, 1, -0.5f * eRb.z);
  // f = m a . b3 (the commanded thrust's adjoint is Mb.f)
  V3 ab = (b.m * Mb.f) * b3;
  b3b = b3b + (b.m * Mb.f) * S.a;
  Rcb[2] = Rcb[2] + b3b;
  // b1d = b2d x b3d
  V3 b2db = Rdb[1], b3db = Rdb[2];
  cross_bwd(S.b2d, S.b3d, Rdb[0], b2db, b3db);
  // b2d = c / |c|,  c = b3d x b1c
  const V3 cb = normalize_bwd(S.b2d, S.cn, b2db);
  b3db = b3db + cross(S.b1c, cb);
  // b3d = a / |a| (constant e3 in the degenerate case |a| = 0)
  if (S.an > 1e-9f) ab = ab + normalize_bwd(S.b3d, S.an, b3db);
  // a = -k_x (p - p_d) - k_v v + g e3
  const V3 ex = x.p - pd;
  pb = pb - V3{g.kx.x * ab.x, g.kx.y * ab.y, g.kx.z * ab.z};
  vb = vb - V3{g.kv.x * ab.x, g.kv.y * ab.y, g.kv.z * ab.z};
  gb.kx = gb.kx - V3{ex.x * ab.x, ex.y * ab.y, ex.z * ab.z};
  gb.kv = gb.kv - V3{x.v.x * ab.x, x.v.y * ab.y, x.v.z * ab.z};
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

// Forward recording: n_steps steps from the fleet state, checkpoint (state,
// motors) every K steps into ckpt[s][13 + 8][n], loss per env, final state
// written back, saturation flag per env.
template <int NROT>
__device__ void record_one(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  const uint32_t n = ab.n;
  Xs<NROT> x;
  load_x(ab.state, ab.motors, n, i, x);
  store_x(ab.ckpt, ab.ckpt + 13 * n, n, i, x);  // checkpoint 0 keeps the raw (possibly non-unit) q_0
  normalize(x.q);
  const Body b = body_at(ab.body, n, i);
  const Gains g = gains_of(P);
  const V3 pd = {ab.targets[i], ab.targets[n + i], ab.targets[2 * n + i]};
  float spsi, cpsi;
  sincosf(ab.targets[3 * n + i], &spsi, &cpsi);
  const V3 goal = {ab.p_goal[i], ab.p_goal[n + i], ab.p_goal[2 * n + i]};
  float loss = 0.f;
  bool saturated = false;
  for (int t = 0; t < ab.n_steps; ++t) {
    if (t > 0 && t % ab.K == 0)
      store_x(ab.ckpt + (size_t)(t / ab.K) * 21 * n, ab.ckpt + (size_t)(t / ab.K) * 21 * n + 13 * n, n, i, x);
    Step<NROT> S;
    Xs<NROT> xn;
    forward_step(x, pd, cpsi, spsi, b, g, P, S, xn);
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

__global__ void __launch_bounds__(128) k_record(AdjointBuffers ab, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ab.n) return;
  const int nr = rotors_of(ab, i);
  if (nr == 4) record_one<4>(ab, P, i);
  else if (nr == 6) record_one<6>(ab, P, i);
  else record_one<8>(ab, P, i);
}

template <int NROT>
__device__ void adjoint_one(const AdjointBuffers& ab, const StepParams& P, uint32_t i) {
  const uint32_t n = ab.n;
  const Body b = body_at(ab.body, n, i);
  const Gains g = gains_of(P);
  const V3 pd = {ab.targets[i], ab.targets[n + i], ab.targets[2 * n + i]};
  float spsi, cpsi;
  sincosf(ab.targets[3 * n + i], &spsi, &cpsi);
  const V3 goal = {ab.p_goal[i], ab.p_goal[n + i], ab.p_goal[2 * n + i]};
  const float wgt = ab.loss_weights ? ab.loss_weights[i] : 1.f;
  Adj<NROT> lam;
  lam.p = lam.v = lam.w = {0.f, 0.f, 0.f};
  lam.q = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < NROT; ++k) lam.u[k] = 0.f;
  GainAdj gb;
  gb.kx = gb.kv = gb.kR = gb.kW = {0.f, 0.f, 0.f};
  const int H = ab.n_steps, K = ab.K;
  const int n_seg = (H + K - 1) / K;
  for (int seg = n_seg - 1; seg >= 0; --seg) {
    const int t0 = seg * K;
    const int len = H - t0 < K ? H - t0 : K;
    Xs<NROT> x;
    load_x(ab.ckpt + (size_t)seg * 21 * n, ab.ckpt + (size_t)seg * 21 * n + 13 * n, n, i, x);
    if (seg == 0) normalize(x.q);
    // recompute the segment's step-start states into the tape
    for (int t = 0; t < len; ++t) {
      store_x(ab.tape + (size_t)t * 21 * n, ab.tape + (size_t)t * 21 * n + 13 * n, n, i, x);
      Step<NROT> S;
      Xs<NROT> xn;
      forward_step(x, pd, cpsi, spsi, b, g, P, S, xn);
      x = xn;
    }
    // reverse sweep
    for (int t = len - 1; t >= 0; --t) {
      load_x(ab.tape + (size_t)t * 21 * n, ab.tape + (size_t)t * 21 * n + 13 * n, n, i, x);
      Step<NROT> S;
      Xs<NROT> xn;
      forward_step(x, pd, cpsi, spsi, b, g, P, S, xn);
      // this step's loss term acts on x_{t+1}
      const V3 e = xn.p - goal;
      lam.p = lam.p + (2.f * ab.w_pos * wgt) * e;
      lam.w = lam.w + (2.f * ab.w_omega * wgt) * xn.w;
      backward_step(x, pd, cpsi, spsi, b, g, P, S, lam, gb);
    }
  }
  // the kernel normalised q_0 at load: q_hat = q0 / |q0|
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
  const float v12[12] = {gb.kx.x, gb.kx.y, gb.kx.z, gb.kv.x, gb.kv.y, gb.kv.z,
                         gb.kR.x, gb.kR.y, gb.kR.z, gb.kW.x, gb.kW.y, gb.kW.z};
#pragma unroll
  for (int k = 0; k < 12; ++k) gg[k * n + i] = v12[k];
}

__global__ void __launch_bounds__(128) k_adjoint(AdjointBuffers ab, StepParams P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ab.n) return;
  const int nr = rotors_of(ab, i);
  if (nr == 4) adjoint_one<4>(ab, P, i);
  else if (nr == 6) adjoint_one<6>(ab, P, i);
  else adjoint_one<8>(ab, P, i);
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

__global__ void __launch_bounds__(256) k_count_non_position(const uint8_t* modes, uint32_t n, uint32_t* count) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = i < n && modes[i] != kModePosition;
  const unsigned m = __ballot_sync(0xFFFFFFFFu, bad);
  if ((threadIdx.x & 31u) == 0 && m) atomicAdd(count, (uint32_t)__popc(m));
}

}  // namespace

cudaError_t launch_count_non_position(const uint8_t* modes, uint32_t n, uint32_t* count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_count_non_position<<<(n + 255) / 256, 256, 0, st>>>(modes, n, count);
  return cudaGetLastError();
}

cudaError_t launch_record(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st) {
  k_record<<<(ab.n + 127) / 128, 128, 0, st>>>(ab, P);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st) {
  k_adjoint<<<(ab.n + 127) / 128, 128, 0, st>>>(ab, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g1(kReduceParts, 12);
  k_reduce_partial<<<g1, kRedThreads, 0, st>>>(ab.grad_gains_env, ab.n, ab.partial, kReduceParts);
  k_reduce_final<<<12, kRedThreads, 0, st>>>(ab.partial, kReduceParts, ab.grad_gains);
  return cudaGetLastError();
}

}  // namespace agk
