// ag_api.cu — the core extern "C" entry points declared in include/ag.h:
// context, inputs and outputs, steps, resets and the controller stage.
// (ag_api_task.cu: depth images and the reach task; ag_api_adjoint.cu: the
// differentiable rollout; ag_api_noalloc.cu: the allocation-free step.)
//
// Host side of libaerialgb: argument validation, device buffers, the
// per-context sticky error state, the FP64 rotor-allocation matrices, and
// the stream-ordered copies and launches. Nothing here computes a vehicle
// state; every step of the simulation runs in the kernels.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ctx_internal.h"

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace agh {

void set_global_error(const std::string& msg) { g_create_error = msg; }

ag_status fail_invalid(ag_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return AG_ERR_INVALID;
}

ag_status check_cuda(ag_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return AG_OK;
  ctx->failed = true;
  ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
  return AG_ERR_CUDA;
}

// Rotor allocation matrices in FP64. Rotor i of n sits at angle
// beta_0 + 360 i / n degrees (beta_0 = 45 for a quad "X", 30 hexa, 22.5 octo)
// at radius `arm`, thrusts along body +z and spins alternately (+, -, ...):
// its column of A is (1, y_i, -x_i, s_i k_yaw). A^+ = A^T (A A^T)^-1.
void rotor_matrices(int n, double arm, double k_yaw, float A[4][8], float Ap[8][4]) {
  const double pi = 3.14159265358979323846;
  const double start = n == 4 ? 45.0 : (n == 6 ? 30.0 : 22.5);
  double a[4][8] = {};
  for (int i = 0; i < n; ++i) {
    double beta = (start + 360.0 * i / n) * pi / 180.0;
    a[0][i] = 1.0;
    a[1][i] = arm * std::sin(beta);
    a[2][i] = -arm * std::cos(beta);
    a[3][i] = (i % 2 == 0 ? 1.0 : -1.0) * k_yaw;
  }
  // M = A A^T, then solve M X = I by Gauss-Jordan with partial pivoting
  double m[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += a[r][k] * a[c][k];
      m[r][c] = s;
      m[r][c + 4] = r == c ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[p][c])) p = r;
    for (int k = 0; k < 8; ++k) std::swap(m[c][k], m[p][k]);
    double d = m[c][c];
    for (int k = 0; k < 8; ++k) m[c][k] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      double f = m[r][c];
      for (int k = 0; k < 8; ++k) m[r][k] -= f * m[c][k];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) A[r][c] = (float)a[r][c];
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[k][i] * m[k][j + 4];
      Ap[i][j] = i < n ? (float)s : 0.f;
    }
}

}  // namespace agh

namespace {

__global__ void k_fill_rows(float* dst, uint32_t n, float v0, float v1, float v2, float v3, int rows) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[4] = {v0, v1, v2, v3};
  for (int r = 0; r < rows; ++r) dst[(size_t)r * n + i] = v[r];
}

// Precondition checks of ag_set_body and ag_set_obstacles: each counts the
// entries that break them into *bad (one atomic per offending entry).
__device__ __host__ inline bool body_ok(float v) { return v > 0.f && v < 3.0e38f; }
__device__ __host__ inline bool box_ok(const float f[10]) {
  for (int k = 0; k < 3; ++k)
    if (!(f[k] > -3.0e38f && f[k] < 3.0e38f) || !body_ok(f[3 + k])) return false;
  const float q2 = f[6] * f[6] + f[7] * f[7] + f[8] * f[8] + f[9] * f[9];
  return q2 > 1.f - 1e-4f && q2 < 1.f + 1e-4f;  // a unit quaternion (also rejects NaN)
}

__global__ void k_count_bad_body(const float* body, size_t count, uint32_t* bad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && !body_ok(body[i])) atomicAdd(bad, 1u);
}

__global__ void k_count_bad_boxes(const float* boxes, uint32_t n, uint32_t n_obs, uint32_t* bad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * n_obs) return;
  const size_t k = i / n, e = i % n;
  float f[10];
  for (int r = 0; r < 10; ++r) f[r] = boxes[(k * 10 + r) * n + e];
  if (!box_ok(f)) atomicAdd(bad, 1u);
}

}  // namespace

namespace agh {

const char* validate(const ag_config* c) {
  if (!c) return "config is NULL";
  if (c->n_envs == 0) return "n_envs must be >= 1";
  if (c->n_envs > AG_MAX_ENVS) return "n_envs must be <= AG_MAX_ENVS (2^28)";
  if (c->substeps_per_step == 0 || c->substeps_per_step > 65536) return "substeps_per_step must be in 1..65536";
  if (c->record_every > 65536) return "record_every must be <= 65536";
  if (c->integrator > 1) return "integrator must be 0 (semi-implicit Euler) or 1 (RK4)";
  if (c->n_obstacles > AG_MAX_OBSTACLES) return "n_obstacles exceeds AG_MAX_OBSTACLES";
  if ((uint64_t)c->n_quad + c->n_hexa + c->n_octo != c->n_envs) return "n_quad + n_hexa + n_octo must equal n_envs";
  if (!(c->dt > 0.f) || !std::isfinite(c->dt)) return "dt must be > 0";
  if (!(c->motor_tau >= 0.f)) return "motor_tau must be >= 0";
  if (!(c->drag >= 0.f)) return "drag must be >= 0";
  if (!(c->sphere_r >= 0.f)) return "sphere_r must be >= 0";
  if (!(c->u_max > 0.f)) return "u_max must be > 0";
  if (!(c->arm > 0.f)) return "arm must be > 0";
  if (!(c->k_yaw > 0.f)) return "k_yaw must be > 0";
  if (!(c->mass > 0.f) || !(c->inertia[0] > 0.f) || !(c->inertia[1] > 0.f) || !(c->inertia[2] > 0.f))
    return "mass and inertia must be > 0";
  return "";
}

}  // namespace agh

namespace {

size_t buffer_bytes(const ag_config* c) {
  size_t n = c->n_envs;
  size_t per = sizeof(float) * (13 + 8 + 4 + 4 + 4 + 4) + sizeof(uint32_t) * 4 + 3 /* modes, collided, hits */ + 1;
  return n * per + (size_t)c->n_obstacles * 10 * n * sizeof(float) +
         agk::box_pair_elems(n, c->n_obstacles) * sizeof(float2) + sizeof(uint32_t) + sizeof(unsigned long long);
}

}  // namespace

agk::StepParams agk::step_params_for(const ag_config& c, uint64_t seed) {
  agk::StepParams P;
  for (int i = 0; i < 3; ++i) {
    P.kx[i] = c.kx[i]; P.kv[i] = c.kv[i]; P.kR[i] = c.kR[i]; P.kW[i] = c.kW[i];
  }
  for (int t = 0; t < 3; ++t) agh::rotor_matrices(t == 0 ? 4 : (t == 1 ? 6 : 8), c.arm, c.k_yaw, P.A[t], P.Ap[t]);
  const double h = (double)c.dt / c.substeps_per_step;
  P.h = (float)h;
  P.alpha = c.motor_tau > 0.f ? (float)(1.0 - std::exp(-h / (double)c.motor_tau)) : 1.f;
  P.drag = c.drag;
  P.r2 = c.sphere_r * c.sphere_r;
  P.u_max = c.u_max;
  P.seed_lo = (uint32_t)(seed & 0xFFFFFFFFu);
  P.seed_hi = (uint32_t)(seed >> 32);
  P.exact_tests = 0;
  agk::pair_rotor_matrices(P);
  return P;
}

namespace agh {

agk::StepParams step_params(const ag_ctx* ctx) {
  agk::StepParams P;
  const ag_config& c = ctx->cfg;
  for (int i = 0; i < 3; ++i) {
    P.kx[i] = c.kx[i]; P.kv[i] = c.kv[i]; P.kR[i] = c.kR[i]; P.kW[i] = c.kW[i];
  }
  std::memcpy(P.A, ctx->A, sizeof(P.A));
  std::memcpy(P.Ap, ctx->Ap, sizeof(P.Ap));
  const double h = (double)c.dt / c.substeps_per_step;
  P.h = (float)h;
  P.alpha = c.motor_tau > 0.f ? (float)(1.0 - std::exp(-h / (double)c.motor_tau)) : 1.f;
  P.drag = c.drag;
  P.r2 = c.sphere_r * c.sphere_r;
  P.u_max = c.u_max;
  P.seed_lo = (uint32_t)(ctx->seed & 0xFFFFFFFFu);
  P.seed_hi = (uint32_t)(ctx->seed >> 32);
  P.exact_tests = 0;
  agk::pair_rotor_matrices(P);
  return P;
}

ag_status enter(ag_ctx* ctx) {
  if (!ctx) return AG_ERR_INVALID;
  if (ctx->failed) return AG_ERR_STATE;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return check_cuda(ctx, e, "cudaSetDevice");
  ctx->err.clear();
  return AG_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes pa;
  const bool dev = cudaPointerGetAttributes(&pa, p) == cudaSuccess &&
                   (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  return dev;
}

}  // namespace agh

namespace {

using namespace agh;

void free_adjoint(ag_ctx* ctx) {
  agk::AdjointBuffers& a = ctx->adj;
  void* ptrs[] = {(void*)a.p_goal, a.ckpt, a.tape, a.loss, a.saturated, (void*)a.loss_weights, a.grad_x0,
                  a.grad_gains_env, a.grad_targets, a.partial, a.grad_gains};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

void free_all(ag_ctx* ctx) {
  free_adjoint(ctx);
  if (ctx->cam_ids) cudaFree(ctx->cam_ids);
  if (ctx->depth_stage) cudaFree(ctx->depth_stage);
  if (ctx->live_dev) cudaFree(ctx->live_dev);
  if (ctx->eval_state) cudaFree(ctx->eval_state);
  if (ctx->check_dev) cudaFree(ctx->check_dev);
  if (ctx->reach_goals) cudaFree(ctx->reach_goals);
  if (ctx->reach_steps) cudaFree(ctx->reach_steps);
  agk::FleetBuffers& f = ctx->fb;
  void* ptrs[] = {f.state, f.motors, f.body, f.modes, f.targets, f.boxes, f.epoch, f.collided, f.reset_ids,
                  f.n_reset, f.tests_run, f.cmd, f.wrench, f.resets, f.hits, f.order, f.boxes_slot, ctx->mask_dev,
                  ctx->order_scratch, f.slot_of, (void*)f.box_rand};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// Number of entries of a device array that break a setter's precondition
// (counted by `launch` into ctx->check_dev; synchronises).
template <class Launch>
ag_status count_bad_on_device(ag_ctx* ctx, Launch launch, uint32_t* bad) {
  cudaStream_t st = ctx->stream;
  ag_status s = check_cuda(ctx, cudaMemsetAsync(ctx->check_dev, 0, sizeof(uint32_t), st), "clear check");
  if (s == AG_OK) s = check_cuda(ctx, launch(st), "check launch");
  if (s == AG_OK)
    s = check_cuda(ctx, cudaMemcpyAsync(bad, ctx->check_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "copy check");
  if (s == AG_OK) s = check_cuda(ctx, cudaStreamSynchronize(st), "synchronize");
  return s;
}

}  // namespace

using namespace agh;

extern "C" {

int ag_abi_version(void) { return AG_ABI_VERSION; }

void ag_config_default(ag_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_envs = 1024;
  c->substeps_per_step = 1;
  c->integrator = AG_INTEG_SIE;
  c->n_obstacles = 0;
  c->n_quad = 1024;
  c->dt = 0.01f;
  c->motor_tau = 0.03f;
  c->drag = 0.f;
  c->sphere_r = 0.2f;
  c->u_max = 5.f;
  c->arm = 0.13f;
  c->k_yaw = 0.016f;
  c->mass = 0.75f;
  c->inertia[0] = 0.007f; c->inertia[1] = 0.007f; c->inertia[2] = 0.012f;
  const float kx[3] = {2.f, 2.f, 3.f}, kv[3] = {2.f, 2.f, 2.f}, kR[3] = {1.2f, 1.2f, 0.6f}, kW[3] = {0.2f, 0.2f, 0.1f};
  for (int i = 0; i < 3; ++i) { c->kx[i] = kx[i]; c->kv[i] = kv[i]; c->kR[i] = kR[i]; c->kW[i] = kW[i]; }
  c->seed = 1;
  c->hbm_budget_bytes = 0;
}

ag_status ag_create(const ag_config* cfg, void* cuda_stream, ag_ctx** out) {
  if (!out) return fail_invalid(nullptr, "out is NULL");
  *out = nullptr;
  std::string why = validate(cfg);
  if (!why.empty()) return fail_invalid(nullptr, why);
  if (cfg->hbm_budget_bytes && buffer_bytes(cfg) > cfg->hbm_budget_bytes) {
    g_create_error = "buffers need " + std::to_string(buffer_bytes(cfg)) + " bytes, budget is " +
                     std::to_string(cfg->hbm_budget_bytes);
    return AG_ERR_OOM;
  }
  ag_ctx* ctx = new (std::nothrow) ag_ctx();
  if (!ctx) { g_create_error = "host allocation failed"; return AG_ERR_OOM; }
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->seed = cfg->seed;
  std::memset(&ctx->fb, 0, sizeof(ctx->fb));
  ctx->mask_dev = nullptr;
  ctx->order_scratch = nullptr;
  std::memset(&ctx->adj, 0, sizeof(ctx->adj));
  ctx->adj_ckpt_cap = 0;
  ctx->adj_tape_cap = 0;
  ctx->adj_recorded = false;
  ctx->cam_ids = nullptr;
  ctx->depth_stage = nullptr;
  ctx->depth_stage_cap = 0;
  ctx->eval_state = nullptr;
  ctx->check_dev = nullptr;
  ctx->reach_goals = nullptr;
  ctx->reach_steps = nullptr;
  ctx->reach_active = false;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    g_create_error = "no CUDA device";
    delete ctx;
    return AG_ERR_CUDA;
  }
  for (int t = 0; t < 3; ++t) rotor_matrices(t == 0 ? 4 : (t == 1 ? 6 : 8), cfg->arm, cfg->k_yaw, ctx->A[t], ctx->Ap[t]);
  const size_t n = cfg->n_envs;
  agk::FleetBuffers& f = ctx->fb;
  f.n = cfg->n_envs; f.n_quad = cfg->n_quad; f.n_hexa = cfg->n_hexa; f.n_octo = cfg->n_octo;
  f.n_obs = cfg->n_obstacles;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = alloc(ctx, &f.state, 13 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.motors, 8 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.body, 4 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.modes, n);
  if (e == cudaSuccess) e = alloc(ctx, &f.targets, 4 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.boxes, (size_t)cfg->n_obstacles * 10 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.boxes_slot, agk::box_pair_elems(n, cfg->n_obstacles));
  if (e == cudaSuccess) e = alloc(ctx, &f.epoch, n);
  if (e == cudaSuccess) e = alloc(ctx, &f.collided, n);
  if (e == cudaSuccess) e = alloc(ctx, &f.reset_ids, n);
  if (e == cudaSuccess) e = alloc(ctx, &f.n_reset, 1);
  if (e == cudaSuccess) e = alloc(ctx, &f.tests_run, 1);
  if (e == cudaSuccess) e = alloc(ctx, &f.cmd, 4 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.wrench, 4 * n);
  if (e == cudaSuccess) e = alloc(ctx, &f.resets, n);
  if (e == cudaSuccess) e = alloc(ctx, &f.hits, n);
  if (e == cudaSuccess) e = alloc(ctx, &ctx->mask_dev, n);
  if (e == cudaSuccess) e = alloc(ctx, &ctx->check_dev, 1);
  if (e == cudaSuccess) e = alloc(ctx, &f.order, n);
  if (e == cudaSuccess && cfg->n_obstacles) e = alloc(ctx, &f.slot_of, n);
  if (e == cudaSuccess) e = alloc(ctx, &ctx->order_scratch, agk::order_scratch_words(cfg->n_envs));
  if (e != cudaSuccess) {
    g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return AG_ERR_OOM;
  }
  cudaStream_t st = ctx->stream;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.state, 0, 13 * n * sizeof(float), st);
  if (e == cudaSuccess) { k_fill_rows<<<grid, 256, 0, st>>>(f.state + 6 * n, (uint32_t)n, 1.f, 0, 0, 0, 1); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaMemsetAsync(f.motors, 0, 8 * n * sizeof(float), st);
  if (e == cudaSuccess) {
    k_fill_rows<<<grid, 256, 0, st>>>(f.body, (uint32_t)n, cfg->mass, cfg->inertia[0], cfg->inertia[1], cfg->inertia[2], 4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(f.modes, AG_MODE_WRENCH, n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.targets, 0, 4 * n * sizeof(float), st);
  if (e == cudaSuccess && f.boxes) e = cudaMemsetAsync(f.boxes, 0, (size_t)cfg->n_obstacles * 10 * n * sizeof(float), st);
  if (e == cudaSuccess && f.boxes_slot)
    e = cudaMemsetAsync(f.boxes_slot, 0, agk::box_pair_elems(n, cfg->n_obstacles) * sizeof(float2), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.epoch, 0, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.collided, 0, n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.n_reset, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.tests_run, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = agk::launch_build_order(f, ctx->order_scratch, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    g_create_error = std::string("initialisation failed: ") + cudaGetErrorString(e);
    free_all(ctx);
    delete ctx;
    return AG_ERR_CUDA;
  }
  *out = ctx;
  return AG_OK;
}

ag_status ag_destroy(ag_ctx* ctx) {
  if (!ctx) return AG_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return AG_OK;
}

ag_status ag_set_commands(ag_ctx* ctx, const uint8_t* modes, const float* targets) {
  agk::NvtxRange range("ag_set_commands");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const size_t n = ctx->cfg.n_envs;
  if (modes) {
    s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.modes, modes, n, cudaMemcpyDefault, ctx->stream), "copy modes");
    if (s != AG_OK) return s;
    s = check_cuda(ctx, agk::launch_build_order(ctx->fb, ctx->order_scratch, ctx->stream), "build order");
    if (s != AG_OK) return s;
  }
  if (targets)
    s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.targets, targets, 4 * n * sizeof(float), cudaMemcpyDefault,
                                        ctx->stream), "copy targets");
  return s;
}

ag_status ag_set_obstacles(ag_ctx* ctx, const float* boxes) {
  agk::NvtxRange range("ag_set_obstacles");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!boxes) return fail_invalid(ctx, "boxes is NULL");
  if (ctx->cfg.n_obstacles == 0) return AG_OK;
  const uint32_t n = ctx->cfg.n_envs, n_obs = ctx->cfg.n_obstacles;
  const size_t count = (size_t)n_obs * 10 * n;
  uint32_t bad = 0;
  if (on_device(boxes)) {
    s = count_bad_on_device(ctx, [&](cudaStream_t st) {
      const size_t items = (size_t)n * n_obs;
      k_count_bad_boxes<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(boxes, n, n_obs, ctx->check_dev);
      return cudaGetLastError();
    }, &bad);
    if (s != AG_OK) return s;
  } else {
    for (size_t k = 0; k < n_obs; ++k)
      for (size_t e = 0; e < n; ++e) {
        float f[10];
        for (int r = 0; r < 10; ++r) f[r] = boxes[(k * 10 + r) * n + e];
        bad += box_ok(f) ? 0u : 1u;
      }
  }
  if (bad) return fail_invalid(ctx, "boxes: finite centres, half-extents > 0 and unit quaternions required");
  s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.boxes, boxes, count * sizeof(float), cudaMemcpyDefault, ctx->stream),
                 "copy boxes");
  if (s != AG_OK) return s;
  return check_cuda(ctx, agk::launch_permute_boxes(ctx->fb, ctx->stream), "permute boxes");
}

ag_status ag_get_obstacles(ag_ctx* ctx, float* boxes) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!boxes) return fail_invalid(ctx, "boxes is NULL");
  const size_t count = (size_t)ctx->cfg.n_obstacles * 10 * ctx->cfg.n_envs;
  if (count == 0) return AG_OK;
  return check_cuda(ctx, cudaMemcpyAsync(boxes, ctx->fb.boxes, count * sizeof(float), cudaMemcpyDefault, ctx->stream),
                    "copy boxes out");
}

ag_status ag_set_obstacle_randomization(ag_ctx* ctx, const float env_min[3], const float env_max[3],
                                        const ag_box_randomization* per_box) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  agk::FleetBuffers& f = ctx->fb;
  const uint32_t n_obs = ctx->cfg.n_obstacles;
  if (!per_box) {
    f.box_rand = nullptr;
    return AG_OK;
  }
  if (n_obs == 0) return fail_invalid(ctx, "the context has no obstacles");
  if (!env_min || !env_max) return fail_invalid(ctx, "env_min and env_max are required");
  const float pi = 3.14159265358979f;
  std::vector<agk::BoxRandDev> spec(n_obs);
  for (uint32_t k = 0; k < n_obs; ++k) {
    const ag_box_randomization& r = per_box[k];
    agk::BoxRandDev& d = spec[k];
    for (int i = 0; i < 3; ++i) {
      if (!(r.pos_min[i] >= 0.f && r.pos_max[i] <= 1.f && r.pos_min[i] <= r.pos_max[i]))
        return fail_invalid(ctx, "position fractions must satisfy 0 <= pos_min <= pos_max <= 1");
      if (!(r.euler_min[i] >= -pi && r.euler_max[i] <= pi && r.euler_min[i] <= r.euler_max[i]))
        return fail_invalid(ctx, "Euler bounds must satisfy -pi <= euler_min <= euler_max <= pi");
      if ((r.lock & (1u << (3 + i))) && !(r.fixed[3 + i] >= -pi && r.fixed[3 + i] <= pi))
        return fail_invalid(ctx, "held angles must lie in [-pi, pi]");
      if (!(env_min[i] <= env_max[i])) return fail_invalid(ctx, "env_min must not exceed env_max");
      d.pos_min[i] = r.pos_min[i]; d.pos_max[i] = r.pos_max[i];
      d.euler_min[i] = r.euler_min[i]; d.euler_max[i] = r.euler_max[i];
      d.env_min[i] = env_min[i]; d.env_max[i] = env_max[i];
    }
    d.lock = r.lock;
    for (int i = 0; i < 6; ++i) d.fixed[i] = r.fixed[i];
  }
  if (!f.box_rand) {
    agk::BoxRandDev* p = nullptr;
    if ((s = alloc_or_oom(ctx, &p, n_obs, "the obstacle spec")) != AG_OK) return s;
    f.box_rand = p;
  }
  return check_cuda(ctx, cudaMemcpy((void*)f.box_rand, spec.data(), n_obs * sizeof(agk::BoxRandDev),
                                    cudaMemcpyHostToDevice), "copy obstacle spec");
}

ag_status ag_set_body(ag_ctx* ctx, const float* body) {
  agk::NvtxRange range("ag_set_body");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!body) return fail_invalid(ctx, "body is NULL");
  const size_t count = 4 * (size_t)ctx->cfg.n_envs;
  uint32_t bad = 0;
  if (on_device(body)) {
    s = count_bad_on_device(ctx, [&](cudaStream_t st) {
      k_count_bad_body<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(body, count, ctx->check_dev);
      return cudaGetLastError();
    }, &bad);
    if (s != AG_OK) return s;
  } else {
    for (size_t i = 0; i < count; ++i) bad += body_ok(body[i]) ? 0u : 1u;
  }
  if (bad) return fail_invalid(ctx, "body: masses and inertias must be finite and > 0");
  return check_cuda(ctx, cudaMemcpyAsync(ctx->fb.body, body, count * sizeof(float), cudaMemcpyDefault, ctx->stream),
                    "copy body");
}

static ag_status step_common(ag_ctx* ctx, uint32_t n_substeps, bool fused) {
  agk::NvtxRange range(fused ? "ag_step" : "ag_step_plain");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const uint32_t sps = ctx->cfg.substeps_per_step;
  if (n_substeps == 0 || n_substeps % sps != 0)
    return fail_invalid(ctx, "n_substeps must be a positive multiple of substeps_per_step");
  if (n_substeps / sps > (uint32_t)INT32_MAX) return fail_invalid(ctx, "at most 2^31 - 1 steps per call");
  agk::StepParams P = step_params(ctx);
  const int n_steps = (int)(n_substeps / sps);
  cudaError_t e = fused ? agk::launch_fused_step(ctx->fb, P, (int)ctx->cfg.integrator, n_steps, (int)sps, ctx->stream)
                        : agk::launch_plain_step(ctx->fb, P, (int)ctx->cfg.integrator, n_steps, (int)sps, ctx->stream);
  return check_cuda(ctx, e, fused ? "fused step launch" : "plain step launch");
}

ag_status ag_step(ag_ctx* ctx, uint32_t n_substeps) { return step_common(ctx, n_substeps, true); }
ag_status ag_step_plain(ag_ctx* ctx, uint32_t n_substeps) { return step_common(ctx, n_substeps, false); }

ag_status ag_inject_failure(ag_ctx* ctx, const char* why) {
  if (!ctx) return AG_ERR_INVALID;
  ctx->failed = true;
  ctx->err = why ? why : "injected failure";
  return AG_OK;
}

ag_status ag_eval_controller(ag_ctx* ctx, const float* state, float* wrench) {
  agk::NvtxRange range("ag_eval_controller");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!wrench) return fail_invalid(ctx, "wrench must be non-NULL");
  const size_t n = ctx->cfg.n_envs;
  cudaStream_t st = ctx->stream;
  agk::FleetBuffers fb = ctx->fb;
  if (state) {
    if (!ctx->eval_state &&
        (s = alloc_or_oom(ctx, &ctx->eval_state, 13 * n, "the controller states")) != AG_OK) return s;
    if ((s = check_cuda(ctx, cudaMemcpyAsync(ctx->eval_state, state, 13 * n * sizeof(float), cudaMemcpyDefault, st),
                        "copy controller states")) != AG_OK) return s;
    fb.state = ctx->eval_state;
  }
  // the unfused path's command scratch receives the result
  if ((s = check_cuda(ctx, agk::launch_controller(fb, step_params(ctx), st), "controller launch")) != AG_OK) return s;
  return check_cuda(ctx, cudaMemcpyAsync(wrench, fb.cmd, 4 * n * sizeof(float), cudaMemcpyDefault, st),
                    "copy wrench out");
}

ag_status ag_reset(ag_ctx* ctx, const uint8_t* mask, uint64_t seed) {
  agk::NvtxRange range("ag_reset");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const uint8_t* mask_dev = nullptr;
  if (mask) {
    s = check_cuda(ctx, cudaMemcpyAsync(ctx->mask_dev, mask, ctx->cfg.n_envs, cudaMemcpyDefault, ctx->stream),
                   "copy mask");
    if (s != AG_OK) return s;
    mask_dev = ctx->mask_dev;
  }
  ctx->seed = seed;
  return check_cuda(ctx, agk::launch_reset(ctx->fb, mask_dev, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
                                           ctx->stream), "reset launch");
}

ag_status ag_get_state(ag_ctx* ctx, float* state, uint8_t* collided, uint32_t* reset_ids, uint32_t* n_reset) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const size_t n = ctx->cfg.n_envs;
  cudaStream_t st = ctx->stream;
  if (state && (s = check_cuda(ctx, cudaMemcpyAsync(state, ctx->fb.state, 13 * n * sizeof(float), cudaMemcpyDefault, st),
                               "copy state out")) != AG_OK) return s;
  if (collided && (s = check_cuda(ctx, cudaMemcpyAsync(collided, ctx->fb.collided, n, cudaMemcpyDefault, st),
                                  "copy collided out")) != AG_OK) return s;
  if (reset_ids && (s = check_cuda(ctx, cudaMemcpyAsync(reset_ids, ctx->fb.reset_ids, n * sizeof(uint32_t),
                                                        cudaMemcpyDefault, st), "copy reset ids out")) != AG_OK) return s;
  if (n_reset) {
    uint32_t tmp = 0;
    if ((s = check_cuda(ctx, cudaMemcpyAsync(&tmp, ctx->fb.n_reset, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                        "copy reset count out")) != AG_OK) return s;
    if ((s = check_cuda(ctx, cudaStreamSynchronize(st), "synchronize")) != AG_OK) return s;
    *n_reset = tmp;
  }
  return AG_OK;
}

ag_status ag_get_motors(ag_ctx* ctx, float* motors, uint32_t* epoch) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const size_t n = ctx->cfg.n_envs;
  if (motors && (s = check_cuda(ctx, cudaMemcpyAsync(motors, ctx->fb.motors, 8 * n * sizeof(float), cudaMemcpyDefault,
                                                     ctx->stream), "copy motors out")) != AG_OK) return s;
  if (epoch) s = check_cuda(ctx, cudaMemcpyAsync(epoch, ctx->fb.epoch, n * sizeof(uint32_t), cudaMemcpyDefault,
                                                ctx->stream), "copy epoch out");
  return s;
}

ag_status ag_set_state(ag_ctx* ctx, const float* state, const float* motors, const uint32_t* epoch) {
  agk::NvtxRange range("ag_set_state");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!state) return fail_invalid(ctx, "state is NULL");
  const size_t n = ctx->cfg.n_envs;
  if ((s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.state, state, 13 * n * sizeof(float), cudaMemcpyDefault, ctx->stream),
                      "copy state in")) != AG_OK) return s;
  if (motors && (s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.motors, motors, 8 * n * sizeof(float), cudaMemcpyDefault,
                                                     ctx->stream), "copy motors in")) != AG_OK) return s;
  if (epoch) s = check_cuda(ctx, cudaMemcpyAsync(ctx->fb.epoch, epoch, n * sizeof(uint32_t), cudaMemcpyDefault,
                                                ctx->stream), "copy epoch in");
  return s;
}

ag_status ag_synchronize(ag_ctx* ctx) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "synchronize");
}

ag_status ag_get_config(const ag_ctx* ctx, ag_config* out) {
  if (!ctx || !out) return AG_ERR_INVALID;
  *out = ctx->cfg;
  return AG_OK;
}

const char* ag_last_error(const ag_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"

