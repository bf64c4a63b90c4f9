// ag_api_adjoint.cu — extern "C" entry points of the differentiable rollout
// (ag_set_gains, ag_rollout_loss, ag_backward).
#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "ctx_internal.h"

using namespace agh;

// ---------------------------------------------------------------------------
// Differentiable rollout: gains, recorded forward, adjoint.
namespace {

// Grows the adjoint buffers for a record of n_steps steps with interval K.
ag_status ensure_adjoint(ag_ctx* ctx, int n_steps, int K) {
  agk::AdjointBuffers& a = ctx->adj;
  const size_t n = ctx->cfg.n_envs;
  const size_t n_ckpt = (size_t)(n_steps + K - 1) / K;
  cudaError_t e = cudaSuccess;
  if (!a.loss) {
    float* pg = nullptr; float* lw = nullptr;
    if (e == cudaSuccess) e = alloc(ctx, &pg, 3 * n);
    if (e == cudaSuccess) e = alloc(ctx, &a.loss, n);
    if (e == cudaSuccess) e = alloc(ctx, &a.saturated, n);
    if (e == cudaSuccess) e = alloc(ctx, &lw, n);
    if (e == cudaSuccess) e = alloc(ctx, &a.grad_x0, 13 * n);
    if (e == cudaSuccess) e = alloc(ctx, &a.grad_gains_env, 12 * n);
    if (e == cudaSuccess) e = alloc(ctx, &a.grad_targets, 4 * n);
    if (e == cudaSuccess) e = alloc(ctx, &a.partial, 12 * (size_t)agk::kReduceParts);
    if (e == cudaSuccess) e = alloc(ctx, &a.grad_gains, 12);
    a.p_goal = pg;
    a.loss_weights = lw;
    if (e != cudaSuccess) { cudaGetLastError(); ctx->err = "adjoint buffers do not fit"; return AG_ERR_OOM; }
  }
  if (n_ckpt > ctx->adj_ckpt_cap) {
    if (a.ckpt) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(a.ckpt);
      a.ckpt = nullptr;
      ctx->bytes -= ctx->adj_ckpt_cap * 21 * n * sizeof(float);
    }
    e = alloc(ctx, &a.ckpt, n_ckpt * 21 * n);
    if (e != cudaSuccess) { cudaGetLastError(); ctx->adj_ckpt_cap = 0; ctx->err = "checkpoints do not fit"; return AG_ERR_OOM; }
    ctx->adj_ckpt_cap = n_ckpt;
  }
  // The tape of step-start states: the whole horizon when it fits (within
  // hbm_budget_bytes when one is set), so that the backward pass can
  // recompute every segment in parallel; else one segment of K steps.
  const size_t step_bytes = 21 * n * sizeof(float);
  const size_t held = (size_t)ctx->adj_tape_cap * step_bytes;
  auto free_tape = [&]() {
    if (a.tape) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(a.tape);
      a.tape = nullptr;
      ctx->bytes -= held;
    }
    ctx->adj_tape_cap = 0;
  };
  if ((size_t)ctx->adj_tape_cap < (size_t)n_steps) {
    const size_t full_bytes = (size_t)n_steps * step_bytes;
    const uint64_t budget = ctx->cfg.hbm_budget_bytes;
    if (budget == 0 || ctx->bytes - held + full_bytes <= budget) {
      free_tape();
      if (alloc(ctx, &a.tape, (size_t)n_steps * 21 * n) == cudaSuccess) {
        ctx->adj_tape_cap = n_steps;
      } else {
        cudaGetLastError();  // an out-of-memory cudaMalloc leaves no sticky error
        a.tape = nullptr;
      }
    }
  }
  a.full_tape = (size_t)ctx->adj_tape_cap >= (size_t)n_steps ? 1 : 0;
  if (!a.full_tape && K > ctx->adj_tape_cap) {
    free_tape();
    e = alloc(ctx, &a.tape, (size_t)K * 21 * n);
    if (e != cudaSuccess) { cudaGetLastError(); ctx->adj_tape_cap = 0; ctx->err = "tape does not fit"; return AG_ERR_OOM; }
    ctx->adj_tape_cap = K;
  }
  return AG_OK;
}

}  // namespace

extern "C" ag_status ag_set_gains(ag_ctx* ctx, const float* gains12) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!gains12) return fail_invalid(ctx, "gains is NULL");
  float g[12];
  if ((s = check_cuda(ctx, cudaMemcpy(g, gains12, sizeof(g), cudaMemcpyDefault), "copy gains")) != AG_OK) return s;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(g[i])) return fail_invalid(ctx, "gains must be finite");
  for (int i = 0; i < 3; ++i) {
    ctx->cfg.kx[i] = g[i]; ctx->cfg.kv[i] = g[3 + i]; ctx->cfg.kR[i] = g[6 + i]; ctx->cfg.kW[i] = g[9 + i];
  }
  return AG_OK;
}

extern "C" ag_status ag_rollout_loss(ag_ctx* ctx, uint32_t n_steps, float w_pos, float w_omega, const float* p_goal,
                                     float* loss, uint8_t* saturated) {
  agk::NvtxRange range("ag_rollout_loss");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const ag_config& c = ctx->cfg;
  if (c.integrator != AG_INTEG_SIE || c.substeps_per_step != 1 || c.n_obstacles != 0) {
    ctx->err = "the differentiable rollout needs semi-implicit Euler, 1 substep per step and no obstacles";
    return AG_ERR_UNSUPPORTED;
  }
  if (n_steps == 0 || n_steps > (1u << 30) || !p_goal || !loss)
    return fail_invalid(ctx, "n_steps must be in 1..2^30; p_goal and loss are required");
  const size_t n = c.n_envs;
  const int K = c.record_every ? (int)c.record_every : 32;
  if ((s = ensure_adjoint(ctx, (int)n_steps, K)) != AG_OK) return s;
  agk::AdjointBuffers& a = ctx->adj;
  if ((s = check_cuda(ctx, cudaMemcpyAsync((void*)a.p_goal, p_goal, 3 * n * sizeof(float), cudaMemcpyDefault,
                                           ctx->stream), "copy goals")) != AG_OK) return s;
  a.state = ctx->fb.state; a.motors = ctx->fb.motors; a.body = ctx->fb.body; a.targets = ctx->fb.targets;
  a.modes = ctx->fb.modes;
  a.n = c.n_envs; a.n_quad = c.n_quad; a.n_hexa = c.n_hexa; a.n_octo = c.n_octo;
  a.n_steps = (int)n_steps; a.K = K; a.w_pos = w_pos; a.w_omega = w_omega;
  ctx->adj_P = step_params(ctx);
  ctx->adj_recorded = false;
  if ((s = check_cuda(ctx, agk::launch_record(a, ctx->adj_P, ctx->stream), "record launch")) != AG_OK) return s;
  ctx->adj_recorded = true;
  if ((s = check_cuda(ctx, cudaMemcpyAsync(loss, a.loss, n * sizeof(float), cudaMemcpyDefault, ctx->stream),
                      "copy loss out")) != AG_OK) return s;
  if (saturated)
    s = check_cuda(ctx, cudaMemcpyAsync(saturated, a.saturated, n, cudaMemcpyDefault, ctx->stream), "copy flags out");
  return s;
}

extern "C" ag_status ag_backward(ag_ctx* ctx, const float* loss_weights, float* grad_x0, float* grad_gains,
                                 float* grad_gains_per_env, float* grad_targets) {
  agk::NvtxRange range("ag_backward");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!ctx->adj_recorded) {
    ctx->err = "ag_backward needs a rollout recorded by ag_rollout_loss";
    return AG_ERR_STATE;
  }
  if (!grad_x0 && !grad_gains && !grad_gains_per_env && !grad_targets) return AG_OK;
  agk::AdjointBuffers a = ctx->adj;
  const size_t n = ctx->cfg.n_envs;
  if (loss_weights) {
    if ((s = check_cuda(ctx, cudaMemcpyAsync((void*)a.loss_weights, loss_weights, n * sizeof(float),
                                             cudaMemcpyDefault, ctx->stream), "copy weights")) != AG_OK) return s;
  } else {
    a.loss_weights = nullptr;
  }
  if ((s = check_cuda(ctx, agk::launch_adjoint(a, ctx->adj_P, ctx->stream), "adjoint launch")) != AG_OK) return s;
  cudaStream_t st = ctx->stream;
  if (grad_x0 && (s = check_cuda(ctx, cudaMemcpyAsync(grad_x0, a.grad_x0, 13 * n * sizeof(float), cudaMemcpyDefault,
                                                      st), "copy grad x0")) != AG_OK) return s;
  if (grad_gains && (s = check_cuda(ctx, cudaMemcpyAsync(grad_gains, a.grad_gains, 12 * sizeof(float),
                                                         cudaMemcpyDefault, st), "copy grad gains")) != AG_OK) return s;
  if (grad_gains_per_env && (s = check_cuda(ctx, cudaMemcpyAsync(grad_gains_per_env, a.grad_gains_env,
                                                                  12 * n * sizeof(float), cudaMemcpyDefault, st),
                                             "copy per-env grad gains")) != AG_OK) return s;
  if (grad_targets)
    s = check_cuda(ctx, cudaMemcpyAsync(grad_targets, a.grad_targets, 4 * n * sizeof(float), cudaMemcpyDefault, st),
                   "copy grad targets");
  return s;
}

