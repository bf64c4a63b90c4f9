// adjoint_internal.h — launch interface of the differentiable rollout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fleet_device.cuh"

namespace agk {

constexpr int kReduceParts = 256;  // first-level blocks of the gain-gradient reduction

// Device buffers of one recorded rollout and its adjoint. Checkpoint s holds
// the state (13 rows) and motors (8 rows) at step s*K as [21][n]; the tape
// holds step-start states in the same layout: every step of the horizon when
// full_tape is set, else one segment's K steps.
struct AdjointBuffers {
  float* state;                // [13][n] fleet state (advanced by the record)
  float* motors;               // [8][n]
  const float* body;           // [4][n]
  const uint8_t* modes;        // [n] command mode per env (values above 3 act as a wrench)
  const float* targets;        // [4][n] command targets
  const float* p_goal;         // [3][n]
  float* ckpt;                 // [S][21][n]
  float* tape;                 // [n_steps][21][n] (full_tape) or [K][21][n]
  float* loss;                 // [n]
  uint8_t* saturated;          // [n] some motor hit a clamp during the record
  const float* loss_weights;   // [n] upstream gradient of each env's loss (NULL = 1)
  float* grad_x0;              // [13][n]
  float* grad_gains_env;       // [12][n]
  float* grad_targets;         // [4][n]
  float* partial;              // [12][kReduceParts]
  float* grad_gains;           // [12]
  uint32_t n, n_quad, n_hexa, n_octo;
  int n_steps, K;
  int full_tape;               // 1: the tape spans the whole horizon (recomputed by k_tape)
  float w_pos, w_omega;
};

cudaError_t launch_record(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st);
cudaError_t launch_adjoint(const AdjointBuffers& ab, const StepParams& P, cudaStream_t st);

}  // namespace agk
