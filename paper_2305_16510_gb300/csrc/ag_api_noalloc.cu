// ag_api_noalloc.cu — the allocation-free unfused step (ag_step_plain_noalloc).
#include <cstdint>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "ctx_internal.h"

using namespace agh;

// ---------------------------------------------------------------------------
// Allocation-free unfused step (ag_step_plain_noalloc).
//
// The unfused path needs four scratch arrays between its stage kernels (the
// commanded and the realised wrench, the per-step hit bytes and the per-call
// reset counters). Here they live in one file-scope device array sized for
// AG_NOALLOC_MAX_ENVS environments, so the call never allocates: every GPU
// that loads this library holds the array until the process exits, and every
// call on that GPU reuses it.
#include <mutex>

namespace {

constexpr size_t kNoallocN = AG_NOALLOC_MAX_ENVS;
constexpr size_t kNoallocOffCmd = 0;
constexpr size_t kNoallocOffWrench = kNoallocOffCmd + 4 * kNoallocN * sizeof(float);
constexpr size_t kNoallocOffResets = kNoallocOffWrench + 4 * kNoallocN * sizeof(float);
constexpr size_t kNoallocOffHits = kNoallocOffResets + kNoallocN * sizeof(uint32_t);
constexpr size_t kNoallocBytes = kNoallocOffHits + kNoallocN;  // 2,424,832 bytes for 65,536 envs
static_assert(kNoallocOffWrench % 256 == 0 && kNoallocOffResets % 256 == 0 && kNoallocOffHits % 256 == 0,
              "scratch sub-arrays must stay 256-byte aligned");

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_base[kNoallocMaxDevices] = {};

void noalloc_error(char* buf, size_t len, const char* msg) {
  if (buf && len) std::snprintf(buf, len, "%s", msg);
}


}  // namespace

// The scratch itself. Host code must not use this name as an address: it is a
// host-side stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

extern "C" ag_status ag_step_plain_noalloc(const ag_config* cfg, void* cuda_stream, uint32_t n_substeps,
                                           uint64_t seed, float* state, float* motors, const float* body,
                                           const uint8_t* modes, const float* targets, const float* boxes,
                                           uint32_t* epoch, uint8_t* collided, uint32_t* reset_ids,
                                           uint32_t* n_reset, char* err, size_t err_len) {
  noalloc_error(err, err_len, "");
  const char* why = validate(cfg);
  if (why[0] != '\0') {
    noalloc_error(err, err_len, why);
    return AG_ERR_INVALID;
  }
  if (cfg->n_envs > AG_NOALLOC_MAX_ENVS) {
    noalloc_error(err, err_len, "n_envs exceeds AG_NOALLOC_MAX_ENVS (65536): use a context (ag_create) instead");
    return AG_ERR_INVALID;
  }
  if (n_substeps == 0 || n_substeps % cfg->substeps_per_step != 0 ||
      n_substeps / cfg->substeps_per_step > (uint32_t)INT32_MAX) {
    noalloc_error(err, err_len, "n_substeps must be a positive multiple of substeps_per_step (at most 2^31 - 1 steps)");
    return AG_ERR_INVALID;
  }
  const void* required[] = {state, motors, body, modes, targets, epoch, collided, reset_ids, n_reset};
  for (const void* p : required)
    if (!p || !on_device(p)) {
      noalloc_error(err, err_len, "every buffer must be a non-NULL device pointer");
      return AG_ERR_INVALID;
    }
  if (cfg->n_obstacles > 0 && (!boxes || !on_device(boxes))) {
    noalloc_error(err, err_len, "boxes must be a device pointer when n_obstacles > 0");
    return AG_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    noalloc_error(err, err_len, "no usable CUDA device");
    return AG_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        noalloc_error(err, err_len, cudaGetErrorString(e));
        return AG_ERR_CUDA;
      }
      g_noalloc_base[dev] = static_cast<unsigned char*>(p);
    }
    base = g_noalloc_base[dev];
  }
  agk::FleetBuffers fb;
  std::memset(&fb, 0, sizeof(fb));
  fb.state = state;
  fb.motors = motors;
  fb.body = const_cast<float*>(body);
  fb.modes = const_cast<uint8_t*>(modes);
  fb.targets = const_cast<float*>(targets);
  fb.boxes = const_cast<float*>(boxes);
  fb.epoch = epoch;
  fb.collided = collided;
  fb.reset_ids = reset_ids;
  fb.n_reset = n_reset;
  fb.cmd = reinterpret_cast<float*>(base + kNoallocOffCmd);
  fb.wrench = reinterpret_cast<float*>(base + kNoallocOffWrench);
  fb.resets = reinterpret_cast<uint32_t*>(base + kNoallocOffResets);
  fb.hits = base + kNoallocOffHits;
  fb.n = cfg->n_envs;
  fb.n_quad = cfg->n_quad;
  fb.n_hexa = cfg->n_hexa;
  fb.n_octo = cfg->n_octo;
  fb.n_obs = cfg->n_obstacles;
  agk::StepParams P;
  for (int i = 0; i < 3; ++i) {
    P.kx[i] = cfg->kx[i]; P.kv[i] = cfg->kv[i]; P.kR[i] = cfg->kR[i]; P.kW[i] = cfg->kW[i];
  }
  for (int t = 0; t < 3; ++t) rotor_matrices(t == 0 ? 4 : (t == 1 ? 6 : 8), cfg->arm, cfg->k_yaw, P.A[t], P.Ap[t]);
  const double h = (double)cfg->dt / cfg->substeps_per_step;
  P.h = (float)h;
  P.alpha = cfg->motor_tau > 0.f ? (float)(1.0 - std::exp(-h / (double)cfg->motor_tau)) : 1.f;
  P.drag = cfg->drag;
  P.r2 = cfg->sphere_r * cfg->sphere_r;
  P.u_max = cfg->u_max;
  P.seed_lo = (uint32_t)(seed & 0xFFFFFFFFu);
  P.seed_hi = (uint32_t)(seed >> 32);
  e = agk::launch_plain_step(fb, P, (int)cfg->integrator, (int)(n_substeps / cfg->substeps_per_step),
                             (int)cfg->substeps_per_step, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    noalloc_error(err, err_len, cudaGetErrorString(e));
    return AG_ERR_CUDA;
  }
  return AG_OK;
}
