// ag_api_noalloc.cu — the allocation-free unfused step (ag_step_plain_noalloc).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>
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

namespace {

constexpr size_t kNoallocN = AG_NOALLOC_MAX_ENVS;
constexpr size_t kNoallocOffCmd = 0;
constexpr size_t kNoallocOffWrench = kNoallocOffCmd + 4 * kNoallocN * sizeof(float);
constexpr size_t kNoallocOffResets = kNoallocOffWrench + 4 * kNoallocN * sizeof(float);
constexpr size_t kNoallocOffHits = kNoallocOffResets + kNoallocN * sizeof(uint32_t);
constexpr size_t kNoallocBytes = kNoallocOffHits + kNoallocN;  // 2,424,832 bytes for 65,536 envs
static_assert(kNoallocOffWrench % 256 == 0 && kNoallocOffResets % 256 == 0 && kNoallocOffHits % 256 == 0,
              "scratch sub-arrays must stay 256-byte aligned");

// The array's device address belongs to the CUDA context that loaded this
// module, not to the device: a host application may make its own driver-API
// context current, and cudaDeviceReset replaces the primary context. So the
// address is looked up again on every call made outside stream capture, and
// remembered per context for calls made while a stream is being captured
// (where a first lookup could load the module into the context).
constexpr int kNoallocMaxContexts = 64;
struct ScratchEntry {
  CUcontext ctx;
  unsigned char* base;
};
std::mutex g_noalloc_mutex;
ScratchEntry g_noalloc_cache[kNoallocMaxContexts] = {};
int g_noalloc_cache_n = 0;
int g_noalloc_cache_next = 0;  // entry replaced when all are taken (round robin)

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

void noalloc_error(char* buf, size_t len, const char* msg) {
  if (buf && len) std::snprintf(buf, len, "%s", msg);
}

// The context current on this thread, through the driver entry point the
// runtime hands out (the library links no libcuda of its own). nullptr on
// failure.
CUcontext current_context() {
  if (!g_ctx_get_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// The device a kernel buffer lives on; -1 for host memory or an unknown
// pointer. Managed memory reports the device it was allocated against.
int device_of(const void* p) {
  cudaPointerAttributes pa;
  int dev = -1;
  if (cudaPointerGetAttributes(&pa, p) == cudaSuccess &&
      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged))
    dev = pa.device;
  cudaGetLastError();
  return dev;
}

}  // namespace

// The scratch itself. Host code must not use this name as an address: it is a
// host-side stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress, in the context that is current for the call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

// Device address of the scratch array in the current context (see above).
ag_status scratch_base(cudaStream_t stream, unsigned char** base, char* err, size_t err_len) {
  CUcontext ctx = current_context();
  if (!ctx) {
    noalloc_error(err, err_len, "no current CUDA context");
    return AG_ERR_CUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    noalloc_error(err, err_len, "cudaStreamIsCapturing failed on the stream");
    return AG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  int slot = -1;
  for (int i = 0; i < g_noalloc_cache_n; ++i)
    if (g_noalloc_cache[i].ctx == ctx) slot = i;
  if (cap != cudaStreamCaptureStatusNone) {
    if (slot < 0) {
      noalloc_error(err, err_len, "the first call in a CUDA context must come before any stream capture");
      return AG_ERR_STATE;
    }
    *base = g_noalloc_cache[slot].base;
    return AG_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    noalloc_error(err, err_len, cudaGetErrorString(e));
    return AG_ERR_CUDA;
  }
  if (slot < 0) {
    if (g_noalloc_cache_n < kNoallocMaxContexts) {
      slot = g_noalloc_cache_n++;
    } else {
      slot = g_noalloc_cache_next;
      g_noalloc_cache_next = (g_noalloc_cache_next + 1) % kNoallocMaxContexts;
    }
    g_noalloc_cache[slot].ctx = ctx;
  }
  g_noalloc_cache[slot].base = static_cast<unsigned char*>(p);
  *base = g_noalloc_cache[slot].base;
  return AG_OK;
}

}  // namespace

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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    noalloc_error(err, err_len, "no usable CUDA device");
    return AG_ERR_CUDA;
  }
  const cudaStream_t stream = (cudaStream_t)cuda_stream;
  if (stream) {
    int sdev = -1;
    if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess || sdev != dev) {
      cudaGetLastError();
      noalloc_error(err, err_len, "the stream does not belong to the current device");
      return AG_ERR_INVALID;
    }
  }
  const void* required[] = {state, motors, body, modes, targets, epoch, collided, reset_ids, n_reset};
  for (const void* p : required)
    if (!p || device_of(p) != dev) {
      noalloc_error(err, err_len, "every buffer must be a non-NULL pointer to memory of the current device");
      return AG_ERR_INVALID;
    }
  if (cfg->n_obstacles > 0 && (!boxes || device_of(boxes) != dev)) {
    noalloc_error(err, err_len, "boxes must point to memory of the current device when n_obstacles > 0");
    return AG_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  const ag_status s = scratch_base(stream, &base, err, err_len);
  if (s != AG_OK) return s;
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
  const agk::StepParams P = agk::step_params_for(*cfg, seed);
  e = agk::launch_plain_step(fb, P, (int)cfg->integrator, (int)(n_substeps / cfg->substeps_per_step),
                             (int)cfg->substeps_per_step, stream);
  if (e != cudaSuccess) {
    noalloc_error(err, err_len, cudaGetErrorString(e));
    return AG_ERR_CUDA;
  }
  return AG_OK;
}
