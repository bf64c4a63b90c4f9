// serve.cu — continuous-batching rollout server (ag_server_* entry points).
//
// Requests are rollouts of independent quadrotor fleets of any size and
// horizon. A persistent host thread runs the loop
//   admit -> launch one chunk for every active request -> retire -> repeat:
//   * admission is FIFO, bounded by the number of slots and by an HBM budget:
//     every request's buffers are carved out of one device slab that the
//     server allocates once at creation (first-fit free list), so admitting
//     and retiring never call cudaMalloc/cudaFree;
//   * all active requests advance together: one launch of k_serve_step covers
//     every environment of every active request for `chunk_steps` steps (or
//     fewer, for a request's last chunk); a request admitted while others are
//     running joins at the next launch and its state stays resident on the
//     device between launches;
//   * a finished request's final state and reset epochs are copied to the
//     host, its slab region is freed, and its latency (completion - submit)
//     is recorded;
//   * the next chunk is enqueued before the host waits for the current one,
//     so the device does not idle while the host retires and admits.
// A request's chunk boundaries are counted from its own first launch, so the
// same request gives bit-identical results alone or in any mix.
// With max_active = 1 the same loop is the one-request-per-launch baseline.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ag.h"
#include "fleet_internal.h"
#include "fleet_sim.cuh"

namespace agk {
namespace {

// One active request as the kernel sees it.
struct ServeDesc {
  FleetBuffers fb;          // its own buffers (quadrotors, boxes in slot order)
  uint32_t seed_lo, seed_hi;
  int steps;                // steps in this launch
  uint32_t block_begin;     // first block of this request in the launch
};

constexpr int kServeBlock = 128;

template <int INTEG, bool DRAG>
__global__ void __launch_bounds__(kServeBlock) k_serve_step(const ServeDesc* __restrict__ table, int n_req,
                                                           StepParams P, int substeps) {
  __shared__ int s_req;
  if (threadIdx.x == 0) {  // last request whose first block is <= this block
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (table[mid].block_begin <= blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_req = lo;
  }
  __syncthreads();
  const ServeDesc& d = table[s_req];
  const uint32_t slot = (blockIdx.x - d.block_begin) * blockDim.x + threadIdx.x;
  if (slot >= d.fb.n || d.steps <= 0) return;
  const uint32_t env = d.fb.order[slot];
  GlobalBoxPairs bx{d.fb.boxes_slot, d.fb.n, slot};
  uint32_t resets = 0, tests = 0;
  bool hit = false;
  simulate<4, INTEG, DRAG>(d.fb, P, env, slot, d.steps, substeps, (int)d.fb.n_obs, bx, d.seed_lo, d.seed_hi, resets,
                           hit, tests);
}

// First-fit allocator over [0, size) with coalescing frees (host bookkeeping
// of the device slab).
class SlabAllocator {
 public:
  explicit SlabAllocator(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        sizes_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto s = sizes_.find(off);
    if (s == sizes_.end()) return;
    size_t bytes = s->second;
    sizes_.erase(s);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  std::unordered_map<size_t, size_t> sizes_;
  size_t used_ = 0;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device bytes one request needs (state, motors, body, targets, modes, epoch,
// collided, reset ids, order, boxes twice, order scratch).
size_t request_bytes(size_t n, size_t n_obs) {
  size_t b = 0;
  b += align256(13 * n * 4) + align256(8 * n * 4) + align256(4 * n * 4) + align256(4 * n * 4);
  b += align256(n) + align256(n * 4) + align256(n) + align256(n * 4) + align256(4) + align256(n * 4);
  b += align256(n_obs * 10 * n * 4) + align256(box_pair_elems(n, n_obs) * 8) +
       align256(order_scratch_words((uint32_t)n) * 4);
  return b;
}

}  // namespace
}  // namespace agk

struct ServeRequest {
  uint64_t id;
  ag_request in;
  std::chrono::steady_clock::time_point t_submit, t_done;
  size_t offset = 0;
  agk::FleetBuffers fb{};
  uint32_t* order_scratch = nullptr;
  uint32_t remaining = 0;
  bool started = false;
  bool done = false;
  ag_status status = AG_OK;
  std::vector<float> final_state;
  std::vector<uint32_t> final_epoch;
};

struct ag_server {
  ag_server_config cfg;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;  // results of retired requests, beside the next chunk
  // two chunks can be in flight: chunk k uses buffer k % 2
  cudaEvent_t chunk_start[2] = {nullptr, nullptr}, chunk_done[2] = {nullptr, nullptr};
  unsigned char* slab = nullptr;
  agk::SlabAllocator* alloc = nullptr;
  agk::ServeDesc* table_host[2] = {nullptr, nullptr};  // pinned
  agk::ServeDesc* table_dev[2] = {nullptr, nullptr};
  agk::StepParams P{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeRequest*> pending;
  std::vector<ServeRequest*> active;
  std::unordered_map<uint64_t, ServeRequest*> all;
  uint64_t next_id = 1;
  bool stop = false;
  bool failed = false;
  std::string err;
  std::thread loop;
  // statistics
  uint64_t launches = 0, completed = 0;
  double vehicle_steps = 0.0;
  double gpu_ms = 0.0;
};

namespace {

using Clock = std::chrono::steady_clock;

void carve(ag_server* s, ServeRequest* r) {
  const size_t n = r->in.n_envs, n_obs = r->in.n_obstacles;
  unsigned char* p = s->slab + r->offset;
  auto take = [&](size_t bytes) {
    unsigned char* q = p;
    p += agk::align256(bytes);
    return q;
  };
  agk::FleetBuffers& f = r->fb;
  std::memset(&f, 0, sizeof(f));
  f.state = (float*)take(13 * n * 4);
  f.motors = (float*)take(8 * n * 4);
  f.body = (float*)take(4 * n * 4);
  f.targets = (float*)take(4 * n * 4);
  f.modes = (uint8_t*)take(n);
  f.epoch = (uint32_t*)take(n * 4);
  f.collided = (uint8_t*)take(n);
  f.reset_ids = (uint32_t*)take(n * 4);
  f.n_reset = (uint32_t*)take(4);
  f.order = (uint32_t*)take(n * 4);
  f.boxes = (float*)take(n_obs * 10 * n * 4);
  f.boxes_slot = (float2*)take(agk::box_pair_elems(n, n_obs) * 8);
  r->order_scratch = (uint32_t*)take(agk::order_scratch_words((uint32_t)n) * 4);
  f.n = (uint32_t)n;
  f.n_quad = (uint32_t)n;
  f.n_obs = (uint32_t)n_obs;
  if (n_obs == 0) { f.boxes = nullptr; f.boxes_slot = nullptr; }
}

__global__ void k_fill_body(float* body, uint32_t n, float m, float jx, float jy, float jz) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  body[i] = m; body[n + i] = jx; body[2 * n + i] = jy; body[3 * n + i] = jz;
}

// Uploads a newly admitted request's inputs and draws its initial states.
cudaError_t start_request(ag_server* s, ServeRequest* r) {
  const ag_request& in = r->in;
  const size_t n = in.n_envs;
  const size_t pitch = in.pitch ? in.pitch : n;
  agk::FleetBuffers& f = r->fb;
  cudaStream_t st = s->stream;
  cudaError_t e = cudaMemcpyAsync(f.modes, in.modes, n, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(f.targets, n * 4, in.targets, pitch * 4, n * 4, 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    if (in.body) {
      e = cudaMemcpy2DAsync(f.body, n * 4, in.body, pitch * 4, n * 4, 4, cudaMemcpyDefault, st);
    } else {
      const ag_config& c = s->cfg.physics;
      k_fill_body<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f.body, (uint32_t)n, c.mass, c.inertia[0],
                                                                c.inertia[1], c.inertia[2]);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && in.n_obstacles)
    e = cudaMemcpy2DAsync(f.boxes, n * 4, in.boxes, pitch * 4, n * 4, (size_t)in.n_obstacles * 10, cudaMemcpyDefault,
                          st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f.epoch, 0, n * 4, st);
  if (e == cudaSuccess) e = agk::launch_reset(f, nullptr, (uint32_t)(in.seed & 0xFFFFFFFFu), (uint32_t)(in.seed >> 32), st);
  if (e == cudaSuccess) e = agk::launch_build_order(f, r->order_scratch, st);
  return e;
}

void fail_server(ag_server* s, cudaError_t e, const char* what) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->failed = true;
  s->err = std::string(what) + ": " + cudaGetErrorString(e);
  for (auto& kv : s->all)
    if (!kv.second->done) { kv.second->done = true; kv.second->status = AG_ERR_CUDA; }
  s->cv_done.notify_all();
}

// A chunk handed to the device and not yet retired.
struct InFlight {
  bool valid = false;
  std::vector<ServeRequest*> finishing;  // requests whose last steps it holds
  double vehicle_steps = 0.0;
};

// The loop keeps the device fed: it enqueues chunk k (after any uploads of
// newly admitted requests) and only then waits for chunk k - 1 and retires
// the requests that finished in it, so the next chunk is already queued
// while the host does its bookkeeping. A retired request's final state is
// copied back then, on a stream of its own, while chunk k runs: its slab
// region is released only after that copy.
void serve_loop(ag_server* s) {
  cudaSetDevice(s->device);
  const int substeps = (int)s->cfg.physics.substeps_per_step;
  const bool rk4 = s->cfg.physics.integrator == AG_INTEG_RK4;
  const bool drag = s->cfg.physics.drag != 0.f;
  const uint32_t chunk = s->cfg.chunk_steps;
  InFlight flight[2];
  for (uint64_t k = 0;; ++k) {
    const int b = (int)(k & 1);
    std::vector<ServeRequest*> admitted, sched;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->pending.empty() && s->active.size() < s->cfg.max_active) {
        ServeRequest* r = s->pending.front();
        if (!s->alloc->alloc(agk::request_bytes(r->in.n_envs, r->in.n_obstacles), &r->offset)) break;
        s->pending.pop_front();
        carve(s, r);
        r->remaining = r->in.n_steps;
        s->active.push_back(r);
        admitted.push_back(r);
      }
      for (ServeRequest* r : s->active)
        if (r->remaining > 0) sched.push_back(r);
      if (sched.empty() && !flight[b ^ 1].valid) {  // nothing to launch and nothing in flight
        if (s->stop) return;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    for (ServeRequest* r : admitted) {
      cudaError_t e = start_request(s, r);
      if (e != cudaSuccess) { fail_server(s, e, "admit"); return; }
      r->started = true;
    }
    // chunk k: one launch for every request with steps left (buffer b was
    // last used by chunk k - 2, retired in the previous iteration)
    cudaError_t e = cudaSuccess;
    if (!sched.empty()) {
      agk::NvtxRange range("serve chunk");
      InFlight& f = flight[b];
      uint32_t blocks = 0;
      for (size_t j = 0; j < sched.size(); ++j) {
        ServeRequest* r = sched[j];
        agk::ServeDesc& d = s->table_host[b][j];
        const uint32_t steps = std::min(chunk, r->remaining);
        r->remaining -= steps;
        if (r->remaining == 0) f.finishing.push_back(r);
        f.vehicle_steps += (double)r->in.n_envs * steps;
        d.fb = r->fb;
        d.seed_lo = (uint32_t)(r->in.seed & 0xFFFFFFFFu);
        d.seed_hi = (uint32_t)(r->in.seed >> 32);
        d.steps = (int)steps;
        d.block_begin = blocks;
        blocks += (r->in.n_envs + agk::kServeBlock - 1) / agk::kServeBlock;
      }
      const int n_req = (int)sched.size();
      e = cudaMemcpyAsync(s->table_dev[b], s->table_host[b], sizeof(agk::ServeDesc) * n_req, cudaMemcpyHostToDevice,
                          s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(s->chunk_start[b], s->stream);
      if (e == cudaSuccess) {
        agk::ServeDesc* t = s->table_dev[b];
        if (rk4) {
          if (drag) agk::k_serve_step<agk::kIntegRK4, true><<<blocks, agk::kServeBlock, 0, s->stream>>>(t, n_req, s->P, substeps);
          else agk::k_serve_step<agk::kIntegRK4, false><<<blocks, agk::kServeBlock, 0, s->stream>>>(t, n_req, s->P, substeps);
        } else {
          if (drag) agk::k_serve_step<agk::kIntegSIE, true><<<blocks, agk::kServeBlock, 0, s->stream>>>(t, n_req, s->P, substeps);
          else agk::k_serve_step<agk::kIntegSIE, false><<<blocks, agk::kServeBlock, 0, s->stream>>>(t, n_req, s->P, substeps);
        }
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(s->chunk_done[b], s->stream);
      if (e != cudaSuccess) { fail_server(s, e, "serve launch"); return; }
      f.valid = true;
    }
    // retire chunk k - 1
    InFlight& prev = flight[b ^ 1];
    if (!prev.valid) continue;
    float ms = 0.f;
    e = cudaEventSynchronize(s->chunk_done[b ^ 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, s->chunk_start[b ^ 1], s->chunk_done[b ^ 1]);
    // the results of the requests that finished in chunk k - 1 (pageable
    // destinations: each copy returns once it is done)
    for (ServeRequest* r : prev.finishing) {
      if (e != cudaSuccess) break;
      const size_t n = r->in.n_envs;
      r->final_state.resize(13 * n);
      r->final_epoch.resize(n);
      e = cudaMemcpyAsync(r->final_state.data(), r->fb.state, 13 * n * 4, cudaMemcpyDeviceToHost, s->copy_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->final_epoch.data(), r->fb.epoch, n * 4, cudaMemcpyDeviceToHost, s->copy_stream);
    }
    if (e == cudaSuccess && !prev.finishing.empty()) e = cudaStreamSynchronize(s->copy_stream);
    if (e != cudaSuccess) { fail_server(s, e, "serve retire"); return; }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->launches += 1;
      s->gpu_ms += ms;
      s->vehicle_steps += prev.vehicle_steps;
      const auto now = Clock::now();
      for (ServeRequest* r : prev.finishing) {
        r->t_done = now;
        r->done = true;
        s->alloc->release(r->offset);
        s->completed += 1;
        s->active.erase(std::find(s->active.begin(), s->active.end(), r));
      }
    }
    if (!prev.finishing.empty()) s->cv_done.notify_all();
    prev = InFlight{};
  }
}

}  // namespace

extern "C" {

void ag_server_config_default(ag_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  ag_config_default(&c->physics);
  c->physics.integrator = AG_INTEG_RK4;
  c->physics.substeps_per_step = 4;
  c->max_active = 1024;
  c->chunk_steps = 50;
  c->hbm_budget_bytes = 40ull << 30;
}

ag_status ag_server_create(const ag_server_config* cfg, ag_server** out) {
  if (!out || !cfg) return AG_ERR_INVALID;
  *out = nullptr;
  if (cfg->max_active == 0 || cfg->max_active > AG_SERVER_MAX_ACTIVE || cfg->chunk_steps == 0 ||
      cfg->chunk_steps > (1u << 30) || cfg->hbm_budget_bytes < (1u << 20) || cfg->physics.substeps_per_step == 0 ||
      cfg->physics.substeps_per_step > 65536 || cfg->physics.integrator > 1 ||
      !(cfg->physics.dt > 0.f) || !(cfg->physics.u_max > 0.f) || !(cfg->physics.mass > 0.f))
    return AG_ERR_INVALID;
  ag_server* s = new (std::nothrow) ag_server();
  if (!s) return AG_ERR_OOM;
  s->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  for (int b = 0; b < 2; ++b) {
    if (e == cudaSuccess) e = cudaEventCreate(&s->chunk_done[b]);
    if (e == cudaSuccess) e = cudaEventCreate(&s->chunk_start[b]);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->table_host[b], sizeof(agk::ServeDesc) * cfg->max_active);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->table_dev[b], sizeof(agk::ServeDesc) * cfg->max_active);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->slab, cfg->hbm_budget_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (s->slab) cudaFree(s->slab);
    for (int b = 0; b < 2; ++b) {
      if (s->table_host[b]) cudaFreeHost(s->table_host[b]);
      if (s->table_dev[b]) cudaFree(s->table_dev[b]);
      if (s->chunk_done[b]) cudaEventDestroy(s->chunk_done[b]);
      if (s->chunk_start[b]) cudaEventDestroy(s->chunk_start[b]);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
    return e == cudaErrorMemoryAllocation ? AG_ERR_OOM : AG_ERR_CUDA;
  }
  s->alloc = new agk::SlabAllocator(cfg->hbm_budget_bytes);
  // launch parameters shared by every request (rotor matrices of the quad)
  s->P = agk::step_params_for(cfg->physics, 0);
  s->loop = std::thread(serve_loop, s);
  *out = s;
  return AG_OK;
}

ag_status ag_server_submit(ag_server* s, const ag_request* req, uint64_t* id) {
  if (!s || !req || !id) return AG_ERR_INVALID;
  if (req->n_envs == 0 || req->n_envs > AG_MAX_ENVS || req->n_steps == 0 || req->n_obstacles > AG_MAX_OBSTACLES ||
      !req->modes || !req->targets ||
      (req->n_obstacles && !req->boxes) || (req->pitch && req->pitch < req->n_envs))
    return AG_ERR_INVALID;
  if (agk::request_bytes(req->n_envs, req->n_obstacles) > s->cfg.hbm_budget_bytes) return AG_ERR_OOM;
  ServeRequest* r = new (std::nothrow) ServeRequest();
  if (!r) return AG_ERR_OOM;
  r->in = *req;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) { delete r; return AG_ERR_STATE; }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  *id = r->id;
  return AG_OK;
}

ag_status ag_server_wait(ag_server* s, uint64_t id, double timeout_s, float* final_state, uint32_t* epoch,
                         double* latency_ms) {
  if (!s) return AG_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return AG_ERR_INVALID;
  ServeRequest* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return AG_ERR_TIMEOUT;
  }
  const ag_status st = r->status;
  if (st == AG_OK) {
    const size_t n = r->in.n_envs;
    if (final_state) std::memcpy(final_state, r->final_state.data(), 13 * n * 4);
    if (epoch) std::memcpy(epoch, r->final_epoch.data(), n * 4);
    if (latency_ms)
      *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  }
  s->all.erase(it);
  delete r;
  return st;
}

ag_status ag_server_get_stats(ag_server* s, ag_server_stats* out) {
  if (!s || !out) return AG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  out->launches = s->launches;
  out->completed = s->completed;
  out->pending = s->pending.size();
  out->active = s->active.size();
  out->vehicle_steps = s->vehicle_steps;
  out->gpu_ms = s->gpu_ms;
  out->hbm_used_bytes = s->alloc->used();
  return s->failed ? AG_ERR_STATE : AG_OK;
}

ag_status ag_server_destroy(ag_server* s) {
  if (!s) return AG_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests still queued are abandoned
    for (ServeRequest* r : s->pending) { r->done = true; r->status = AG_ERR_STATE; }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  if (s->loop.joinable()) s->loop.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->all) delete kv.second;
  delete s->alloc;
  cudaFree(s->slab);
  for (int b = 0; b < 2; ++b) {
    cudaFreeHost(s->table_host[b]);
    cudaFree(s->table_dev[b]);
    cudaEventDestroy(s->chunk_done[b]);
    cudaEventDestroy(s->chunk_start[b]);
  }
  cudaStreamDestroy(s->stream);
  cudaStreamSynchronize(s->copy_stream);
  cudaStreamDestroy(s->copy_stream);
  delete s;
  return AG_OK;
}

}  // extern "C"
