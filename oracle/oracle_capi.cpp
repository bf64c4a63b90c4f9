// oracle_capi.cpp — extern "C" surface of the FP64 oracle for ctypes.
//
// TEST INFRASTRUCTURE ONLY (see aerial_oracle.hpp). Build with
// -ffp-contract=off (the reset sampler is defined in strict binary32).
//
// Layouts (all structure-of-arrays over n environments, row r at r * n):
//   state   double[13][n]  p.xyz, v.xyz, q.wxyz, Omega.xyz
//   motors  double[8][n]   rotor thrusts u_0..u_{n_rot-1} (rest unused)
//   body    double[4][n]   m, J_xx, J_yy, J_zz
//   modes   uint8[n]       0 position, 1 body velocity, 2 attitude+thrust, 3 wrench
//   targets double[4][n]   see orc::controller
//   boxes   double[n_obs][10][n]  centre xyz, half-extents xyz, q wxyz
//   epoch   uint32[n]      reset counter used in the Philox counter
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "aerial_oracle.hpp"
#include "philox_sampler.hpp"
#include "scalars.hpp"

namespace {

using namespace orc;

// Obstacle re-draw on reset: environment bounds and one spec per box (NULL
// when obstacles keep their poses).
struct BoxRandSpec {
  float env_min[3], env_max[3];
  const BoxRand* per_box;  // n_obs entries
};

struct World {
  int32_t n_envs, substeps_per_step, integrator, n_obs;
  int32_t n_quad, n_hexa, n_octo, pad_;
  double dt, motor_tau, drag, sphere_r, u_max, arm, k_yaw;
  double kx[3], kv[3], kR[3], kW[3];
  const BoxRandSpec* box_rand;
};

int rotor_count(const World& w, int env) {
  if (env < w.n_quad) return 4;
  if (env < w.n_quad + w.n_hexa) return 6;
  return 8;
}

double motor_alpha(const World& w) {
  double h = w.dt / w.substeps_per_step;
  return w.motor_tau > 0.0 ? 1.0 - std::exp(-h / w.motor_tau) : 1.0;
}

template <class T> Gains<T> gains_of(const double kx[3], const double kv[3], const double kR[3], const double kW[3]) {
  Gains<T> g;
  g.kx = {T(kx[0]), T(kx[1]), T(kx[2])};
  g.kv = {T(kv[0]), T(kv[1]), T(kv[2])};
  g.kR = {T(kR[0]), T(kR[1]), T(kR[2])};
  g.kW = {T(kW[0]), T(kW[1]), T(kW[2])};
  return g;
}

template <class T> State<T> load_state(const double* s, size_t n, size_t i) {
  State<T> st;
  st.p = {T(s[0 * n + i]), T(s[1 * n + i]), T(s[2 * n + i])};
  st.v = {T(s[3 * n + i]), T(s[4 * n + i]), T(s[5 * n + i])};
  st.q = {T(s[6 * n + i]), T(s[7 * n + i]), T(s[8 * n + i]), T(s[9 * n + i])};
  st.w = {T(s[10 * n + i]), T(s[11 * n + i]), T(s[12 * n + i])};
  return st;
}

void store_state(const State<double>& st, double* s, size_t n, size_t i) {
  double v[13] = {st.p.x, st.p.y, st.p.z, st.v.x, st.v.y, st.v.z, st.q.w, st.q.x, st.q.y, st.q.z,
                  st.w.x, st.w.y, st.w.z};
  for (int r = 0; r < 13; ++r) s[r * n + i] = v[r];
}

// One substep: controller -> allocation/clamp/lag -> integrator.
template <class T>
void substep(const Rotors& rot, int mode, const T tgt[4], const Body<T>& body, const Gains<T>& g, double u_max,
             double alpha, double drag, int integrator, T h, State<T>& s, T u[8]) {
  Wrench<T> cmd = controller(mode, s, tgt, body, g);
  Wrench<T> W = allocate(rot, cmd, u, u_max, alpha);
  s = integrator == 1 ? step_rk4(s, W, body, drag, h) : step_sie(s, W, body, drag, h);
}

// Writes a fresh draw into environment i's state and motors (Sec. V reset).
// `id` is the environment number in the Philox counter (normally i). With a
// box re-draw spec the environment's boxes get new poses (boxes may be NULL
// when n_obs is 0).
void apply_reset(const World& w, double* state, double* motors, const double* body, double* boxes, uint32_t* epoch,
                 size_t n, size_t i, int n_rot, uint64_t seed, uint32_t id) {
  epoch[i] += 1u;
  ResetDraw d = sample_reset_f32(seed, id, epoch[i]);
  double v[13] = {d.p[0], d.p[1], d.p[2], d.v[0], d.v[1], d.v[2], d.q[0], d.q[1], d.q[2], d.q[3], 0.0, 0.0, 0.0};
  for (int r = 0; r < 13; ++r) state[r * n + i] = v[r];
  float hover = hover_thrust_f32((float)body[0 * n + i], n_rot);
  for (int k = 0; k < 8; ++k) motors[k * n + i] = k < n_rot ? (double)hover : 0.0;
  if (w.box_rand && boxes) {
    for (int k = 0; k < w.n_obs; ++k) {
      BoxPose bp = sample_box_pose_f32(seed, id, epoch[i], (uint32_t)k, w.box_rand->per_box[k], w.box_rand->env_min,
                                       w.box_rand->env_max);
      double* bx = boxes + (size_t)k * 10 * n;
      for (int f = 0; f < 3; ++f) bx[f * n + i] = bp.c[f];
      for (int f = 0; f < 4; ++f) bx[(6 + f) * n + i] = bp.q[f];
    }
  }
}

bool env_collides(const World& w, const double* boxes, size_t n, size_t i, Vec3<double> p) {
  bool hit = false;
  for (int b = 0; b < w.n_obs; ++b) {
    const double* bx = boxes + (size_t)b * 10 * n;
    Vec3<double> c = {bx[0 * n + i], bx[1 * n + i], bx[2 * n + i]};
    Vec3<double> h = {bx[3 * n + i], bx[4 * n + i], bx[5 * n + i]};
    Quat<double> q = {bx[6 * n + i], bx[7 * n + i], bx[8 * n + i], bx[9 * n + i]};
    if (sphere_hits_box(p, w.sphere_r, c, h, q)) hit = true;
  }
  return hit;
}

void rollout_range(const World& w, const Rotors rot[3], int n_steps, double* state, double* motors,
                   const double* body, const uint8_t* modes, const double* targets, double* boxes,
                   uint32_t* epoch, uint64_t seed, uint8_t* collided, uint32_t* n_resets, const uint32_t* env_ids,
                   size_t i0, size_t i1) {
  const size_t n = (size_t)w.n_envs;
  const double alpha = motor_alpha(w);
  const double h = w.dt / w.substeps_per_step;
  Gains<double> g = gains_of<double>(w.kx, w.kv, w.kR, w.kW);
  for (size_t i = i0; i < i1; ++i) {
    int n_rot = rotor_count(w, (int)i);
    const Rotors& r = rot[n_rot == 4 ? 0 : (n_rot == 6 ? 1 : 2)];
    Body<double> bd = {body[0 * n + i], {body[1 * n + i], body[2 * n + i], body[3 * n + i]}};
    double tgt[4] = {targets[0 * n + i], targets[1 * n + i], targets[2 * n + i], targets[3 * n + i]};
    State<double> s = load_state<double>(state, n, i);
    double u[8];
    for (int k = 0; k < 8; ++k) u[k] = motors[k * n + i];
    uint8_t any_hit = 0;
    uint32_t resets = 0;
    for (int step = 0; step < n_steps; ++step) {
      for (int ss = 0; ss < w.substeps_per_step; ++ss)
        substep(r, modes[i], tgt, bd, g, w.u_max, alpha, w.drag, w.integrator, h, s, u);
      if (w.n_obs > 0 && env_collides(w, boxes, n, i, s.p)) {
        any_hit = 1;
        resets += 1;
        store_state(s, state, n, i);
        apply_reset(w, state, motors, body, boxes, epoch, n, i, n_rot, seed, env_ids ? env_ids[i] : (uint32_t)i);
        s = load_state<double>(state, n, i);
        for (int k = 0; k < 8; ++k) u[k] = motors[k * n + i];
      }
    }
    store_state(s, state, n, i);
    for (int k = 0; k < 8; ++k) motors[k * n + i] = u[k];
    if (collided) collided[i] = any_hit;
    if (n_resets) n_resets[i] = resets;
  }
}

World world_of(const void* p) {
  World w;
  std::memcpy(&w, p, sizeof(World));
  return w;
}

// Loss of one vehicle over a horizon (the differentiable-rollout objective):
//   L = sum_{t=1..H} ( w_pos |p_t - p_goal|^2 + w_omega |Omega_t|^2 ),
// x_t the state after step t. Gains are inputs so their tangents can be set.
template <class T>
T vehicle_loss(const World& w, const Rotors& rot, int mode, const T tgt_in[4], const Body<T>& body,
               State<T> s, T u[8], const Gains<T>& g, int horizon, const double p_goal[3], double w_pos,
               double w_omega) {
  const double alpha = motor_alpha(w);
  const T h = T(w.dt / w.substeps_per_step);
  T tgt[4] = {tgt_in[0], tgt_in[1], tgt_in[2], tgt_in[3]};
  Vec3<T> goal = {T(p_goal[0]), T(p_goal[1]), T(p_goal[2])};
  T loss = T(0);
  for (int t = 0; t < horizon; ++t) {
    for (int ss = 0; ss < w.substeps_per_step; ++ss)
      substep(rot, mode, tgt, body, g, w.u_max, alpha, w.drag, w.integrator, h, s, u);
    Vec3<T> e = s.p - goal;
    loss = loss + T(w_pos) * dot(e, e) + T(w_omega) * dot(s.w, s.w);
  }
  return loss;
}

}  // namespace

extern "C" {

int orc_abi_version(void) { return 1; }
int orc_world_size(void) { return (int)sizeof(World); }

// Rolls every environment forward n_steps steps in place. Each step is
// substeps_per_step substeps followed, when n_obs > 0, by the sphere-vs-box
// test; an environment that hits any box is reset (epoch + 1, fresh draw).
// collided[i] = 1 if env i hit a box in any step of this call; n_resets[i]
// counts its resets. env_ids (may be NULL) gives the environment number
// each row uses in the Philox counter, so a subset of a larger fleet draws
// the same resets as in the full fleet. Work is split over n_threads host
// threads.
int orc_rollout(const void* world, int n_steps, double* state, double* motors, const double* body,
                const uint8_t* modes, const double* targets, double* boxes, uint32_t* epoch, uint64_t seed,
                uint8_t* collided, uint32_t* n_resets, const uint32_t* env_ids, int n_threads) {
  World w = world_of(world);
  if (w.n_envs <= 0 || w.substeps_per_step <= 0 || n_steps < 0) return 1;
  Rotors rot[3] = {make_rotors(4, w.arm, w.k_yaw), make_rotors(6, w.arm, w.k_yaw), make_rotors(8, w.arm, w.k_yaw)};
  size_t n = (size_t)w.n_envs;
  if (n_threads <= 1) {
    rollout_range(w, rot, n_steps, state, motors, body, modes, targets, boxes, epoch, seed, collided, n_resets, env_ids,
                  0, n);
    return 0;
  }
  std::vector<std::thread> pool;
  size_t chunk = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    size_t i0 = t * chunk, i1 = std::min(n, i0 + chunk);
    if (i0 >= i1) break;
    pool.emplace_back(rollout_range, std::cref(w), rot, n_steps, state, motors, body, modes, targets, boxes, epoch,
                      seed, collided, n_resets, env_ids, i0, i1);
  }
  for (auto& th : pool) th.join();
  return 0;
}

// Resets the environments with mask[i] != 0 (all when mask is NULL):
// epoch + 1, then the Philox draw for (seed, id, epoch) and hover motors,
// id = env_ids[i] (NULL: i), as in orc_rollout.
int orc_reset(const void* world, const uint8_t* mask, uint64_t seed, const double* body, double* state,
              double* motors, uint32_t* epoch, const uint32_t* env_ids, double* boxes) {
  World w = world_of(world);
  size_t n = (size_t)w.n_envs;
  for (size_t i = 0; i < n; ++i)
    if (!mask || mask[i])
      apply_reset(w, state, motors, body, boxes, epoch, n, i, rotor_count(w, (int)i), seed,
                  env_ids ? env_ids[i] : (uint32_t)i);
  return 0;
}

int orc_box_rand_size(void) { return (int)sizeof(BoxRand); }

// Reach-a-setpoint task (Sec. I: robots learn to reach a target setpoint
// through the attitude command interface). Reading of its observation, reward
// and termination, per environment i with goal g_i:
//   obs    = (p - g, v, q (w >= 0 hemisphere), Omega)            13 numbers
//   reward = -crash                                 if the vehicle collided
//            -|p - g| - w_v |v| - w_w |Omega|       otherwise
//   done   = collided  or  |p - g| > max_dist  or  steps >= max_steps
// (a collided vehicle was already re-drawn by the step, so its reward carries
// no distance term; steps counts the episode's steps including this one).
void orc_reach_task(int n, const double* state, const double* goals, const uint8_t* collided, const uint32_t* steps,
                    double w_v, double w_w, double crash, double max_dist, uint32_t max_steps, double* obs,
                    double* reward, uint8_t* done) {
  for (int i = 0; i < n; ++i) {
    double s[13];
    for (int r = 0; r < 13; ++r) s[r] = state[(size_t)r * n + i];
    double e[3] = {s[0] - goals[i], s[1] - goals[(size_t)n + i], s[2] - goals[2 * (size_t)n + i]};
    const double sign = s[6] < 0.0 ? -1.0 : 1.0;
    double o[13] = {e[0], e[1], e[2], s[3], s[4], s[5], sign * s[6], sign * s[7], sign * s[8], sign * s[9],
                    s[10], s[11], s[12]};
    for (int r = 0; r < 13; ++r) obs[(size_t)r * n + i] = o[r];
    const double dist = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    const double speed = std::sqrt(s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    const double rate = std::sqrt(s[10] * s[10] + s[11] * s[11] + s[12] * s[12]);
    reward[i] = collided[i] ? -crash : -dist - w_v * speed - w_w * rate;
    done[i] = (collided[i] || dist > max_dist || steps[i] >= max_steps) ? 1 : 0;
  }
}

// Depth images of n_cams cameras (row-major [cam][H][W]); camera j belongs to
// environment env_ids[j] of a fleet with `n` environments (state double[13][n],
// boxes double[n_obs][10][n]). See ray_box_depth for the camera model.
void orc_render_depth(int n, int n_obs, const double* state, const double* boxes, int n_cams, const uint32_t* env_ids,
                      int W, int H, double hfov, double max_range, const double cam_offset[3], double* out) {
  const double f = 0.5 * W / std::tan(0.5 * hfov);
  for (int j = 0; j < n_cams; ++j) {
    const size_t i = env_ids[j];
    State<double> s = load_state<double>(state, (size_t)n, i);
    Mat3<double> R = quat_to_rot(s.q);
    Vec3<double> o = s.p + matvec(R, Vec3<double>{cam_offset[0], cam_offset[1], cam_offset[2]});
    for (int r = 0; r < H; ++r)
      for (int c = 0; c < W; ++c) {
        Vec3<double> dc = {1.0, -(c + 0.5 - 0.5 * W) / f, -(r + 0.5 - 0.5 * H) / f};
        Vec3<double> d = matvec(R, dc);
        double best = max_range;
        for (int k = 0; k < n_obs; ++k) {
          const double* bx = boxes + (size_t)k * 10 * n;
          double t = ray_box_depth(o, d, Vec3<double>{bx[0 * n + i], bx[1 * n + i], bx[2 * n + i]},
                                   Vec3<double>{bx[3 * n + i], bx[4 * n + i], bx[5 * n + i]},
                                   Quat<double>{bx[6 * n + i], bx[7 * n + i], bx[8 * n + i], bx[9 * n + i]}, max_range);
          if (t < best) best = t;
        }
        out[((size_t)j * H + r) * W + c] = best;
      }
  }
}

// One box pose draw (tests of the sampler): out7 = centre xyz, q wxyz.
void orc_sample_box_pose(uint64_t seed, uint32_t env, uint32_t epoch, uint32_t k, const void* spec,
                         const float env_min[3], const float env_max[3], float out7[7]) {
  BoxRand r;
  std::memcpy(&r, spec, sizeof(r));
  BoxPose b = sample_box_pose_f32(seed, env, epoch, k, r, env_min, env_max);
  for (int i = 0; i < 3; ++i) out7[i] = b.c[i];
  for (int i = 0; i < 4; ++i) out7[3 + i] = b.q[i];
}

// ---- single-function entry points used by the oracle's own pins ----------
void orc_hat(const double a[3], double out[9]) {
  Mat3<double> m = hat(Vec3<double>{a[0], a[1], a[2]});
  for (int i = 0; i < 9; ++i) out[i] = m.a[i / 3][i % 3];
}
void orc_vee(const double m9[9], double out[3]) {
  Mat3<double> m;
  for (int i = 0; i < 9; ++i) m.a[i / 3][i % 3] = m9[i];
  Vec3<double> v = vee(m);
  out[0] = v.x; out[1] = v.y; out[2] = v.z;
}
void orc_quat_to_rot(const double q[4], double out[9]) {
  Mat3<double> m = quat_to_rot(Quat<double>{q[0], q[1], q[2], q[3]});
  for (int i = 0; i < 9; ++i) out[i] = m.a[i / 3][i % 3];
}
void orc_attitude_errors(const double R9[9], const double W[3], const double Rd9[9], const double Wd[3],
                         const double body4[4], const double gains12[12], double eR[3], double eW[3], double M[3]) {
  Mat3<double> R, Rd;
  for (int i = 0; i < 9; ++i) { R.a[i / 3][i % 3] = R9[i]; Rd.a[i / 3][i % 3] = Rd9[i]; }
  Body<double> b = {body4[0], {body4[1], body4[2], body4[3]}};
  Gains<double> g = gains_of<double>(gains12, gains12 + 3, gains12 + 6, gains12 + 9);
  ControlOut<double> out;
  attitude_law(R, Vec3<double>{W[0], W[1], W[2]}, Rd, Vec3<double>{Wd[0], Wd[1], Wd[2]}, b, g, out);
  for (int i = 0; i < 3; ++i) {
    eR[i] = i == 0 ? out.eR.x : (i == 1 ? out.eR.y : out.eR.z);
    eW[i] = i == 0 ? out.eW.x : (i == 1 ? out.eW.y : out.eW.z);
    M[i] = i == 0 ? out.cmd.M.x : (i == 1 ? out.cmd.M.y : out.cmd.M.z);
  }
}
void orc_desired_rate(double phi, double theta, double yaw_rate, double out[3]) {
  Vec3<double> r = desired_rate(phi, theta, yaw_rate);
  out[0] = r.x; out[1] = r.y; out[2] = r.z;
}
// Controller of one vehicle: out_fM = (f, M), plus R_d (row-major), Omega_d,
// e_R and e_Omega of that evaluation.
void orc_controller(int mode, const double state13[13], const double tgt[4], const double body4[4],
                    const double gains12[12], double out_fM[4], double out_Rd[9], double out_Wd[3], double out_eR[3],
                    double out_eW[3]) {
  State<double> s = load_state<double>(state13, 1, 0);
  Body<double> b = {body4[0], {body4[1], body4[2], body4[3]}};
  Gains<double> g = gains_of<double>(gains12, gains12 + 3, gains12 + 6, gains12 + 9);
  ControlOut<double> d;
  Wrench<double> W = controller(mode, s, tgt, b, g, &d);
  out_fM[0] = W.f; out_fM[1] = W.M.x; out_fM[2] = W.M.y; out_fM[3] = W.M.z;
  if (mode == MODE_WRENCH) return;
  for (int i = 0; i < 9; ++i) out_Rd[i] = d.Rd.a[i / 3][i % 3];
  out_Wd[0] = d.Wd.x; out_Wd[1] = d.Wd.y; out_Wd[2] = d.Wd.z;
  out_eR[0] = d.eR.x; out_eR[1] = d.eR.y; out_eR[2] = d.eR.z;
  out_eW[0] = d.eW.x; out_eW[1] = d.eW.y; out_eW[2] = d.eW.z;
}
// Allocation matrix A (4 x n_rot, row-major in a 4x8 block) and A^+ (8x4).
void orc_rotors(int n_rot, double arm, double k_yaw, double A[32], double Ap[32]) {
  Rotors r = make_rotors(n_rot, arm, k_yaw);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) A[i * 8 + j] = j < n_rot ? r.A[i][j] : 0.0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 4; ++j) Ap[i * 4 + j] = i < n_rot ? r.Ap[i][j] : 0.0;
}
// One allocation/clamp/lag update: u (in/out, n_rot entries), returns W.
void orc_allocate(int n_rot, double arm, double k_yaw, const double cmd4[4], double u[8], double u_max,
                  double alpha, double W_out[4]) {
  Rotors r = make_rotors(n_rot, arm, k_yaw);
  Wrench<double> c = {cmd4[0], {cmd4[1], cmd4[2], cmd4[3]}};
  Wrench<double> W = allocate(r, c, u, u_max, alpha);
  W_out[0] = W.f; W_out[1] = W.M.x; W_out[2] = W.M.y; W_out[3] = W.M.z;
}
// One integrator step of length h under a fixed body wrench W (f, M).
void orc_integrate(int integrator, const double state13[13], const double W4[4], const double body4[4], double drag,
                   double h, double out13[13]) {
  State<double> s = load_state<double>(state13, 1, 0);
  Body<double> b = {body4[0], {body4[1], body4[2], body4[3]}};
  Wrench<double> W = {W4[0], {W4[1], W4[2], W4[3]}};
  State<double> r = integrator == 1 ? step_rk4(s, W, b, drag, h) : step_sie(s, W, b, drag, h);
  store_state(r, out13, 1, 0);
}
int orc_sphere_obb(const double p[3], double r, const double box10[10]) {
  return sphere_hits_box(Vec3<double>{p[0], p[1], p[2]}, r, Vec3<double>{box10[0], box10[1], box10[2]},
                         Vec3<double>{box10[3], box10[4], box10[5]},
                         Quat<double>{box10[6], box10[7], box10[8], box10[9]})
             ? 1
             : 0;
}
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox4x32_10(ctr, key, out); }
void orc_sample_reset(uint64_t seed, uint32_t env, uint32_t epoch, float out10[10]) {
  ResetDraw d = sample_reset_f32(seed, env, epoch);
  for (int i = 0; i < 3; ++i) { out10[i] = d.p[i]; out10[3 + i] = d.v[i]; }
  for (int i = 0; i < 4; ++i) out10[6 + i] = d.q[i];
}
float orc_hover_thrust(float m, int n_rot) { return hover_thrust_f32(m, n_rot); }
void orc_sincos_poly(float h, float* s, float* c) { sincos_poly_f32(h, s, c); }
void orc_sincos_turn(uint32_t w, float* c, float* s) { sincos_turn_f32(w, c, s); }
float orc_log_u01(uint32_t w) { return log_u01_f32(w); }

// Algorithmic operation counts of ONE vehicle-step (substeps_per_step
// substeps of the given mode plus one sphere-vs-box test per box of n_obs)
// for a quadrotor near hover: counts = {add, mul, div, sqrt, trans, cmp}.
void orc_count_ops(const void* world, int mode, int n_obs, int n_rot, long long counts[6]) {
  World w = world_of(world);
  Rotors rot = make_rotors(n_rot, w.arm, w.k_yaw);
  Gains<Cnt> g = gains_of<Cnt>(w.kx, w.kv, w.kR, w.kW);
  Body<Cnt> b = {Cnt(0.75), {Cnt(0.007), Cnt(0.007), Cnt(0.012)}};
  State<Cnt> s;
  s.p = {Cnt(0.3), Cnt(-0.2), Cnt(0.1)};
  s.v = {Cnt(0.1), Cnt(0.2), Cnt(-0.1)};
  s.q = {Cnt(0.99), Cnt(0.05), Cnt(-0.08), Cnt(0.1)};
  s.w = {Cnt(0.1), Cnt(-0.2), Cnt(0.05)};
  Cnt u[8];
  for (int k = 0; k < 8; ++k) u[k] = Cnt(1.8);
  Cnt tgt[4];
  if (mode == MODE_POSITION) { tgt[0] = 1.0; tgt[1] = -1.0; tgt[2] = 0.5; tgt[3] = 0.3; }
  else if (mode == MODE_BODY_VEL) { tgt[0] = 0.5; tgt[1] = -0.5; tgt[2] = 0.2; tgt[3] = 0.1; }
  else if (mode == MODE_ATT_THRUST) { tgt[0] = 0.1; tgt[1] = -0.1; tgt[2] = 0.2; tgt[3] = 7.0; }
  else { tgt[0] = 7.0; tgt[1] = 0.0; tgt[2] = 0.0; tgt[3] = 0.0; }
  const double alpha = motor_alpha(w);
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  Cnt h = Cnt(w.dt / w.substeps_per_step);
  for (int ss = 0; ss < w.substeps_per_step; ++ss)
    substep(rot, mode, tgt, b, g, w.u_max, alpha, w.drag, w.integrator, h, s, u);
  Vec3<Cnt> p = s.p;
  for (int k = 0; k < n_obs; ++k) {
    Vec3<Cnt> c = {Cnt(2.0), Cnt(-1.0), Cnt(0.5)};
    Vec3<Cnt> hb = {Cnt(0.5), Cnt(0.4), Cnt(0.3)};
    Quat<Cnt> qb = {Cnt(0.9), Cnt(0.1), Cnt(0.3), Cnt(0.3)};
    sphere_hits_box(p, Cnt(w.sphere_r), c, hb, qb);
  }
  OpCounts oc = op_counts();
  counts[0] = oc.add; counts[1] = oc.mul; counts[2] = oc.div;
  counts[3] = oc.sqrt; counts[4] = oc.trans; counts[5] = oc.cmp;
}

void put_counts(long long out[6]) {
  OpCounts oc = op_counts();
  out[0] = oc.add; out[1] = oc.mul; out[2] = oc.div; out[3] = oc.sqrt; out[4] = oc.trans; out[5] = oc.cmp;
}

// Operation counts of the depth camera (ray_box_depth, orc_render_depth),
// split by what each part is repeated over: `ray` per pixel (its world-frame
// ray R d_c), `box` per (camera, box) pair (box_in_camera), `pair` per
// (pixel, box) pair (ray_slab_depth, for a ray with no zero component that
// hits the box). Each is {add, mul, div, sqrt, trans, cmp}.
void orc_count_depth_ops(long long ray[6], long long box[6], long long pair[6]) {
  const double W = 480.0, H = 270.0, f = 0.5 * W / std::tan(0.5 * 1.5);
  Quat<Cnt> qc = {Cnt(0.9), Cnt(0.1), Cnt(-0.2), Cnt(0.3)};
  Mat3<Cnt> R = quat_to_rot(qc);
  Vec3<Cnt> o = {Cnt(0.1), Cnt(0.2), Cnt(0.3)};
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  const Cnt c = Cnt(100.0), r = Cnt(50.0);
  Vec3<Cnt> dc = {Cnt(1.0), -(c + Cnt(0.5) - Cnt(0.5 * W)) / Cnt(f), -(r + Cnt(0.5) - Cnt(0.5 * H)) / Cnt(f)};
  Vec3<Cnt> d = matvec(R, dc);
  put_counts(ray);
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  BoxInCamera<Cnt> bc = box_in_camera(o, Vec3<Cnt>{Cnt(3.0), Cnt(0.4), Cnt(0.2)},
                                      Quat<Cnt>{Cnt(0.9), Cnt(0.1), Cnt(0.3), Cnt(0.3)});
  put_counts(box);
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  Cnt t = ray_slab_depth(bc, Vec3<Cnt>{Cnt(1.0), Cnt(0.1), Cnt(0.05)}, Vec3<Cnt>{Cnt(0.5), Cnt(0.5), Cnt(0.5)},
                         Cnt(10.0));
  put_counts(pair);
  (void)d; (void)t;
}

void put_rev(long long out[5]) {
  RevCounts rc = rev_counts();
  out[0] = rc.add; out[1] = rc.mul; out[2] = rc.div; out[3] = rc.sqrt; out[4] = rc.trans;
}

// Forward and reverse-mode operation counts of ONE step of the
// differentiable-rollout objective (vehicle_loss over one step: controller
// of `mode`, allocation, clamp, lag, semi-implicit Euler, and the step's loss
// term) for a vehicle near hover with the state, motors, 12 gains and 4
// targets active. fwd = {add, mul, div, sqrt, trans, cmp} of the step; rev =
// {add, mul, div, sqrt, trans} of its adjoint (see CntRev).
void orc_count_reverse_ops(const void* world, int mode, int n_rot, long long fwd[6], long long rev[5]) {
  World w = world_of(world);
  Rotors rot = make_rotors(n_rot, w.arm, w.k_yaw);
  Gains<CntRev> g;
  g.kx = {CntRev(w.kx[0], true), CntRev(w.kx[1], true), CntRev(w.kx[2], true)};
  g.kv = {CntRev(w.kv[0], true), CntRev(w.kv[1], true), CntRev(w.kv[2], true)};
  g.kR = {CntRev(w.kR[0], true), CntRev(w.kR[1], true), CntRev(w.kR[2], true)};
  g.kW = {CntRev(w.kW[0], true), CntRev(w.kW[1], true), CntRev(w.kW[2], true)};
  Body<CntRev> b = {CntRev(0.75), {CntRev(0.007), CntRev(0.007), CntRev(0.012)}};
  State<CntRev> s;
  s.p = {CntRev(0.3, true), CntRev(-0.2, true), CntRev(0.1, true)};
  s.v = {CntRev(0.1, true), CntRev(0.2, true), CntRev(-0.1, true)};
  s.q = {CntRev(0.99, true), CntRev(0.05, true), CntRev(-0.08, true), CntRev(0.1, true)};
  s.w = {CntRev(0.1, true), CntRev(-0.2, true), CntRev(0.05, true)};
  CntRev u[8];
  for (int k = 0; k < 8; ++k) u[k] = CntRev(1.8, true);
  double t4[4];
  if (mode == MODE_POSITION) { t4[0] = 1.0; t4[1] = -1.0; t4[2] = 0.5; t4[3] = 0.3; }
  else if (mode == MODE_BODY_VEL) { t4[0] = 0.5; t4[1] = -0.5; t4[2] = 0.2; t4[3] = 0.1; }
  else if (mode == MODE_ATT_THRUST) { t4[0] = 0.1; t4[1] = -0.1; t4[2] = 0.2; t4[3] = 7.0; }
  else { t4[0] = 7.0; t4[1] = 0.0; t4[2] = 0.0; t4[3] = 0.0; }
  CntRev tgt[4];
  for (int k = 0; k < 4; ++k) tgt[k] = CntRev(t4[k], true);
  const double goal[3] = {0.5, -0.5, 0.2};
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  rev_counts() = RevCounts{0, 0, 0, 0, 0};
  vehicle_loss(w, rot, mode, tgt, b, s, u, g, 1, goal, 1.0, 0.01);
  put_counts(fwd);
  put_rev(rev);
}

// The same counts for one small building block with every input active, to
// check CntRev against counts made by hand: which = 0 dot(a, b) of two
// 3-vectors, 1 quat_normalize(q), 2 cross(a, b).
void orc_count_reverse_primitive(int which, long long fwd[6], long long rev[5]) {
  Vec3<CntRev> a = {CntRev(0.3, true), CntRev(-0.2, true), CntRev(0.1, true)};
  Vec3<CntRev> bb = {CntRev(0.7, true), CntRev(0.4, true), CntRev(-0.5, true)};
  Quat<CntRev> q = {CntRev(0.9, true), CntRev(0.1, true), CntRev(-0.2, true), CntRev(0.3, true)};
  op_counts() = OpCounts{0, 0, 0, 0, 0, 0};
  rev_counts() = RevCounts{0, 0, 0, 0, 0};
  if (which == 0) (void)dot(a, bb);
  else if (which == 1) (void)quat_normalize(q);
  else (void)cross(a, bb);
  put_counts(fwd);
  put_rev(rev);
}

// Loss of one vehicle (see vehicle_loss) in FP64. gains12 = (k_x, k_v, k_R,
// k_Omega) diagonals; state13 / motors (n_rot entries) are the initial state.
double orc_vehicle_loss(const void* world, int n_rot, int mode, const double tgt[4], const double body4[4],
                        const double state13[13], const double motors[8], const double gains12[12], int horizon,
                        const double p_goal[3], double w_pos, double w_omega) {
  World w = world_of(world);
  Rotors rot = make_rotors(n_rot, w.arm, w.k_yaw);
  Body<double> b = {body4[0], {body4[1], body4[2], body4[3]}};
  State<double> s = load_state<double>(state13, 1, 0);
  double u[8];
  for (int k = 0; k < 8; ++k) u[k] = motors[k];
  Gains<double> g = gains_of<double>(gains12, gains12 + 3, gains12 + 6, gains12 + 9);
  return vehicle_loss(w, rot, mode, tgt, b, s, u, g, horizon, p_goal, w_pos, w_omega);
}

// Directional derivative of orc_vehicle_loss along (d_state13, d_gains12,
// d_tgt4), by forward-mode dual numbers; d_tgt4 may be NULL (targets held).
// Returns the loss; *dloss receives the JVP.
double orc_vehicle_loss_jvp(const void* world, int n_rot, int mode, const double tgt[4], const double body4[4],
                            const double state13[13], const double motors[8], const double gains12[12],
                            const double d_state13[13], const double d_gains12[12], const double* d_tgt4,
                            int horizon, const double p_goal[3], double w_pos, double w_omega, double* dloss) {
  World w = world_of(world);
  Rotors rot = make_rotors(n_rot, w.arm, w.k_yaw);
  Body<Dual> b = {Dual(body4[0]), {Dual(body4[1]), Dual(body4[2]), Dual(body4[3])}};
  double sv[13];
  for (int i = 0; i < 13; ++i) sv[i] = state13[i];
  State<Dual> s;
  s.p = {Dual(sv[0], d_state13[0]), Dual(sv[1], d_state13[1]), Dual(sv[2], d_state13[2])};
  s.v = {Dual(sv[3], d_state13[3]), Dual(sv[4], d_state13[4]), Dual(sv[5], d_state13[5])};
  s.q = {Dual(sv[6], d_state13[6]), Dual(sv[7], d_state13[7]), Dual(sv[8], d_state13[8]), Dual(sv[9], d_state13[9])};
  s.w = {Dual(sv[10], d_state13[10]), Dual(sv[11], d_state13[11]), Dual(sv[12], d_state13[12])};
  Dual u[8];
  for (int k = 0; k < 8; ++k) u[k] = Dual(motors[k]);
  Gains<Dual> g;
  g.kx = {Dual(gains12[0], d_gains12[0]), Dual(gains12[1], d_gains12[1]), Dual(gains12[2], d_gains12[2])};
  g.kv = {Dual(gains12[3], d_gains12[3]), Dual(gains12[4], d_gains12[4]), Dual(gains12[5], d_gains12[5])};
  g.kR = {Dual(gains12[6], d_gains12[6]), Dual(gains12[7], d_gains12[7]), Dual(gains12[8], d_gains12[8])};
  g.kW = {Dual(gains12[9], d_gains12[9]), Dual(gains12[10], d_gains12[10]), Dual(gains12[11], d_gains12[11])};
  Dual tg[4];
  for (int k = 0; k < 4; ++k) tg[k] = Dual(tgt[k], d_tgt4 ? d_tgt4[k] : 0.0);
  Dual L = vehicle_loss(w, rot, mode, tg, b, s, u, g, horizon, p_goal, w_pos, w_omega);
  *dloss = L.d;
  return L.v;
}

}  // extern "C"
