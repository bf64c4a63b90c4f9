// ag_api_task.cu — extern "C" entry points of the depth cameras
// (ag_render_depth) and of the reach-a-setpoint task (ag_reach_*).
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "ctx_internal.h"
#include "depth_internal.h"

using namespace agh;

namespace {

// ag_render_depth and its two measurement variants (ag_measure.h): ieee_div
// renders with correctly rounded reciprocals; a non-NULL live_pairs (host)
// renders nothing and receives the number of (pixel, box) pairs the kernel
// would test after culling (the call then synchronises).
ag_status render_depth_impl(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                            const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams, float* depth,
                            int ieee_div, uint64_t* live_pairs) {
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  const uint32_t n = ctx->cfg.n_envs;
  if (width == 0 || height == 0 || (uint64_t)width * height > (1u << 30))
    return fail_invalid(ctx, "image size must be positive and at most 2^30 pixels");
  if (!(hfov > 0.f && hfov < 3.14159f)) return fail_invalid(ctx, "hfov must lie in (0, pi)");
  if (!(max_range > 0.f)) return fail_invalid(ctx, "max_range must be > 0");
  if (n_cams == 0 || (!depth && !live_pairs)) return fail_invalid(ctx, "n_cams must be >= 1 and depth non-NULL");
  if (!env_ids && n_cams > n) return fail_invalid(ctx, "n_cams exceeds n_envs");
  if (env_ids && n_cams > n) return fail_invalid(ctx, "at most n_envs cameras per call");
  cudaStream_t st = ctx->stream;
  const uint32_t* ids_dev = nullptr;
  if (env_ids) {
    if (!on_device(env_ids))
      for (uint32_t j = 0; j < n_cams; ++j)
        if (env_ids[j] >= n) return fail_invalid(ctx, "environment id out of range");
    if (!ctx->cam_ids && (s = alloc_or_oom(ctx, &ctx->cam_ids, n, "the camera ids")) != AG_OK) return s;
    if ((s = check_cuda(ctx, cudaMemcpyAsync(ctx->cam_ids, env_ids, n_cams * sizeof(uint32_t), cudaMemcpyDefault, st),
                        "copy camera ids")) != AG_OK) return s;
    ids_dev = ctx->cam_ids;
  }
  const size_t count = (size_t)n_cams * width * height;
  const bool out_on_device = live_pairs ? true : on_device(depth);
  float* out = depth;
  if (live_pairs && !ctx->live_dev &&
      (s = alloc_or_oom(ctx, &ctx->live_dev, 1, "the live-pair counter")) != AG_OK)
    return s;
  if (!out_on_device) {
    if (count > ctx->depth_stage_cap) {
      if (ctx->depth_stage) { cudaStreamSynchronize(st); cudaFree(ctx->depth_stage); ctx->depth_stage = nullptr; }
      ctx->depth_stage_cap = 0;
      if ((s = alloc_or_oom(ctx, &ctx->depth_stage, count, "the depth staging buffer")) != AG_OK) return s;
      ctx->depth_stage_cap = count;
    }
    out = ctx->depth_stage;
  }
  agk::DepthArgs a;
  a.state = ctx->fb.state;
  a.boxes = ctx->fb.boxes;
  a.env_ids = ids_dev;
  a.out = out;
  a.n = n;
  a.n_obs = ctx->cfg.n_obstacles;
  a.n_cams = n_cams;
  a.width = width;
  a.height = height;
  a.inv_f = (float)(std::tan(0.5 * (double)hfov) / (0.5 * width));
  a.max_range = max_range;
  for (int i = 0; i < 3; ++i) a.offset[i] = cam_offset ? cam_offset[i] : 0.f;
  a.ieee_div = ieee_div;
  a.live_pairs = nullptr;
  if (live_pairs) {
    a.live_pairs = ctx->live_dev;
    if ((s = check_cuda(ctx, cudaMemsetAsync(ctx->live_dev, 0, sizeof(unsigned long long), st),
                        "clear live-pair counter")) != AG_OK) return s;
  }
  if ((s = check_cuda(ctx, agk::launch_render_depth(a, st), "depth launch")) != AG_OK) return s;
  if (live_pairs) {
    unsigned long long v = 0;
    if ((s = check_cuda(ctx, cudaMemcpyAsync(&v, ctx->live_dev, sizeof(v), cudaMemcpyDeviceToHost, st),
                        "copy live-pair count")) != AG_OK) return s;
    if ((s = check_cuda(ctx, cudaStreamSynchronize(st), "synchronize")) != AG_OK) return s;
    *live_pairs = (uint64_t)v;
    return AG_OK;
  }
  if (!out_on_device)
    s = check_cuda(ctx, cudaMemcpyAsync(depth, out, count * sizeof(float), cudaMemcpyDeviceToHost, st), "copy depth out");
  return s;
}

}  // namespace

extern "C" {

ag_status ag_render_depth(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                          const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams, float* depth) {
  agk::NvtxRange range("ag_render_depth");
  return render_depth_impl(ctx, width, height, hfov, max_range, cam_offset, env_ids, n_cams, depth, 0, nullptr);
}

ag_status ag_render_depth_ieee(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                               const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams, float* depth) {
  agk::NvtxRange range("ag_render_depth_ieee");
  return render_depth_impl(ctx, width, height, hfov, max_range, cam_offset, env_ids, n_cams, depth, 1, nullptr);
}

ag_status ag_depth_live_pairs(ag_ctx* ctx, uint32_t width, uint32_t height, float hfov, float max_range,
                              const float* cam_offset, const uint32_t* env_ids, uint32_t n_cams,
                              uint64_t* live_pairs) {
  agk::NvtxRange range("ag_depth_live_pairs");
  if (ctx && !live_pairs) return fail_invalid(ctx, "live_pairs is NULL");
  return render_depth_impl(ctx, width, height, hfov, max_range, cam_offset, env_ids, n_cams, nullptr, 0,
                           live_pairs);
}

void ag_reach_config_default(ag_reach_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->command_mode = AG_MODE_ATT_THRUST;
  const float pi6 = 0.52359878f, mg = 0.75f * 9.81f;
  const float scale[4] = {pi6, pi6, 1.0f, 0.5f * mg}, offset[4] = {0.f, 0.f, 0.f, mg};
  for (int k = 0; k < 4; ++k) {
    c->action_scale[k] = scale[k];
    c->action_offset[k] = offset[k];
  }
  c->w_v = 0.1f;
  c->w_omega = 0.01f;
  c->crash = 10.f;
  c->max_dist = 8.f;
  c->max_steps = 500;
}

ag_status ag_reach_begin(ag_ctx* ctx, const ag_reach_config* cfg, const float* goals) {
  agk::NvtxRange range("ag_reach_begin");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!cfg || !goals) return fail_invalid(ctx, "cfg and goals must be non-NULL");
  if (cfg->command_mode != AG_MODE_ATT_THRUST && cfg->command_mode != AG_MODE_BODY_VEL)
    return fail_invalid(ctx, "command_mode must be AG_MODE_ATT_THRUST or AG_MODE_BODY_VEL");
  if (cfg->max_steps == 0) return fail_invalid(ctx, "max_steps must be >= 1");
  if (!(cfg->w_v >= 0.f && cfg->w_omega >= 0.f && cfg->crash >= 0.f))
    return fail_invalid(ctx, "weights and the crash penalty must be >= 0");
  if (!(cfg->max_dist > 0.f)) return fail_invalid(ctx, "max_dist must be > 0");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(cfg->action_scale[k]) || !std::isfinite(cfg->action_offset[k]))
      return fail_invalid(ctx, "action scale and offset must be finite");
  const size_t n = ctx->cfg.n_envs;
  cudaStream_t st = ctx->stream;
  if (!ctx->reach_goals && (s = alloc_or_oom(ctx, &ctx->reach_goals, 3 * n, "the goals")) != AG_OK)
    return s;
  if (!ctx->reach_steps && (s = alloc_or_oom(ctx, &ctx->reach_steps, n, "the step counters")) != AG_OK)
    return s;
  if ((s = check_cuda(ctx, cudaMemcpyAsync(ctx->reach_goals, goals, 3 * n * sizeof(float), cudaMemcpyDefault, st),
                      "copy goals")) != AG_OK) return s;
  if ((s = check_cuda(ctx, cudaMemsetAsync(ctx->reach_steps, 0, n * sizeof(uint32_t), st), "clear step counters")) !=
      AG_OK) return s;
  if ((s = check_cuda(ctx, cudaMemsetAsync(ctx->fb.modes, (int)cfg->command_mode, n, st), "set modes")) != AG_OK)
    return s;
  if ((s = check_cuda(ctx, agk::launch_build_order(ctx->fb, ctx->order_scratch, st), "build order")) != AG_OK)
    return s;
  ctx->reach = *cfg;
  ctx->reach_active = true;
  return AG_OK;
}

static agk::ReachArgs reach_args(ag_ctx* ctx, const float* actions, float* obs, float* reward, uint8_t* done) {
  agk::ReachArgs a;
  a.fb = ctx->fb;
  a.actions = actions;
  a.goals = ctx->reach_goals;
  a.steps = ctx->reach_steps;
  a.obs = obs;
  a.reward = reward;
  a.done = done;
  const ag_reach_config& c = ctx->reach;
  for (int k = 0; k < 4; ++k) {
    a.scale[k] = c.action_scale[k];
    a.offset[k] = c.action_offset[k];
  }
  a.w_v = c.w_v;
  a.w_omega = c.w_omega;
  a.crash = c.crash;
  a.max_dist = c.max_dist;
  a.max_steps = c.max_steps;
  a.seed_lo = (uint32_t)(ctx->seed & 0xFFFFFFFFu);
  a.seed_hi = (uint32_t)(ctx->seed >> 32);
  return a;
}

ag_status ag_reach_step(ag_ctx* ctx, const float* actions, float* obs, float* reward, uint8_t* done) {
  agk::NvtxRange range("ag_reach_step");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!ctx->reach_active) return AG_ERR_STATE;
  if (!actions || !obs || !reward || !done) return fail_invalid(ctx, "actions, obs, reward and done must be non-NULL");
  if (reinterpret_cast<uintptr_t>(actions) % 16 != 0) return fail_invalid(ctx, "actions must be 16-byte aligned");
  const agk::ReachArgs a = reach_args(ctx, actions, obs, reward, done);
  return check_cuda(ctx, agk::launch_reach_step(a, step_params(ctx), (int)ctx->cfg.integrator,
                                                (int)ctx->cfg.substeps_per_step, ctx->stream), "task step launch");
}

ag_status ag_reach_observe(ag_ctx* ctx, float* obs) {
  agk::NvtxRange range("ag_reach_observe");
  ag_status s = enter(ctx);
  if (s != AG_OK) return s;
  if (!ctx->reach_active) return AG_ERR_STATE;
  if (!obs) return fail_invalid(ctx, "obs must be non-NULL");
  return check_cuda(ctx, agk::launch_reach_observe(reach_args(ctx, nullptr, obs, nullptr, nullptr), ctx->stream),
                    "task observe launch");
}

}  // extern "C"
