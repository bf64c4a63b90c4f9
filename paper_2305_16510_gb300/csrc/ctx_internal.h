// ctx_internal.h — the context behind ag_ctx and the host helpers that the
// C-ABI files (ag_api*.cu) share.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "adjoint_internal.h"
#include "ag.h"
#include "fleet_internal.h"
#include "task_internal.h"

struct ag_ctx {
  ag_config cfg;
  cudaStream_t stream;
  int device;
  agk::FleetBuffers fb;
  uint8_t* mask_dev;         // [n] staging for ag_reset masks
  uint32_t* order_scratch;   // per-block key counts / offsets of the grouping permutation
  uint64_t seed;             // Philox key of collision resets
  bool failed;
  std::string err;
  size_t bytes;              // device bytes held
  float A[3][4][8], Ap[3][8][4];
  // differentiable rollout (allocated at the first ag_rollout_loss)
  agk::AdjointBuffers adj;
  size_t adj_ckpt_cap;       // checkpoints the ckpt buffer holds
  int adj_tape_cap;          // steps the tape holds
  bool adj_recorded;
  agk::StepParams adj_P;     // parameters of the recorded rollout
  // depth rendering staging (allocated on first use, grown as needed)
  uint32_t* cam_ids;         // [n_envs]
  float* depth_stage;        // device staging when the caller's buffer is on the host
  size_t depth_stage_cap;    // floats
  unsigned long long* live_dev;  // [1] live-pair counter of ag_depth_live_pairs (allocated on first use)
  float* eval_state;         // [13][n_envs] states of ag_eval_controller (allocated on first use)
  uint32_t* check_dev;       // [1] count of the setters' precondition checks
  // reach-a-setpoint task (allocated at the first ag_reach_begin)
  ag_reach_config reach;
  float* reach_goals;        // [3][n_envs]
  uint32_t* reach_steps;     // [n_envs]
  bool reach_active;
};

namespace agh {

// AG_ERR_INVALID with a message (ctx NULL: the message of a failed ag_create).
ag_status fail_invalid(ag_ctx* ctx, const std::string& msg);
// Sets the message ag_last_error(NULL) returns (calls without a context).
void set_global_error(const std::string& msg);
// AG_OK for cudaSuccess; else the context becomes failed (sticky) with the message.
ag_status check_cuda(ag_ctx* ctx, cudaError_t e, const char* what);
// Common prologue of every call on a context: NULL ctx, sticky failure, device selection.
ag_status enter(ag_ctx* ctx);
// Launch parameters of the context's config and current reset seed.
agk::StepParams step_params(const ag_ctx* ctx);
// true for device or managed memory (a kernel can read it), false for host memory.
bool on_device(const void* p);
// Rotor allocation matrix A and its pseudo-inverse A^+ in FP64, stored float32.
void rotor_matrices(int n, double arm, double k_yaw, float A[4][8], float Ap[8][4]);
// "" for a valid config, else a static message (no allocation).
const char* validate(const ag_config* c);

// cudaMalloc of count elements, counted against the context's device bytes.
template <class T> cudaError_t alloc(ag_ctx* ctx, T** p, size_t count) {
  if (count == 0) { *p = nullptr; return cudaSuccess; }
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) ctx->bytes += count * sizeof(T);
  return e;
}

// Allocation made on first use of a feature: AG_OK, or AG_ERR_OOM with the
// message "<what> does not fit" and the context left usable (an out-of-memory
// cudaMalloc leaves no sticky error).
template <class T> ag_status alloc_or_oom(ag_ctx* ctx, T** p, size_t count, const char* what) {
  if (alloc(ctx, p, count) == cudaSuccess) return AG_OK;
  cudaGetLastError();
  *p = nullptr;
  ctx->err = std::string(what) + " does not fit";
  return AG_ERR_OOM;
}

}  // namespace agh
