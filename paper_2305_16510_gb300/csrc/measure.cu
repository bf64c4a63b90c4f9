// measure.cu — ag_measure_fp32_peak (include/ag_measure.h): the FP32 FMA
// throughput the CUDA cores reach, to check the derived denominator of the
// fused step's ALU roofline.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ag_measure.h"
#include "ctx_internal.h"

namespace {

constexpr int kChains = 8;   // independent accumulators per thread
constexpr int kRounds = 16;  // FMAs per accumulator per loop iteration
constexpr int kBlock = 256;

// a <- a * b + c on kChains independent chains; b < 1 keeps every value
// bounded (the chains converge to c / (1 - b)), so no special values appear.
__global__ void __launch_bounds__(kBlock) k_fma_scalar(float* sink, uint32_t iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kRounds; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  sink[(size_t)blockIdx.x * kBlock + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) k_fma_packed(float* sink, uint32_t iters, float b, float c) {
  float2 a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, 0.5f * i);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kRounds; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  sink[(size_t)blockIdx.x * kBlock + threadIdx.x] = s;
}

ag_status cuda_fail(cudaError_t e, const char* what) {
  agh::set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
  return AG_ERR_CUDA;
}

}  // namespace

extern "C" ag_status ag_measure_fp32_peak(void* cuda_stream, uint32_t iters, uint32_t reps, ag_fp32_peak* out) {
  if (!out) return agh::fail_invalid(nullptr, "ag_measure_fp32_peak: out is NULL");
  if (iters < 1 || iters > 1000000) return agh::fail_invalid(nullptr, "ag_measure_fp32_peak: iters must be in 1..1000000");
  if (reps < 1 || reps > 100) return agh::fail_invalid(nullptr, "ag_measure_fp32_peak: reps must be in 1..100");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_packed, kBlock, 0);
  if (e != cudaSuccess) return cuda_fail(e, "ag_measure_fp32_peak: device query");
  const uint32_t grid = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
  float* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&sink, (size_t)grid * kBlock * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  double best[2] = {1e30, 1e30};
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    for (uint32_t r = 0; r <= reps && e == cudaSuccess; ++r) {  // r == 0 is the warm-up
      e = cudaEventRecord(t0, st);
      if (kind == 0) k_fma_scalar<<<grid, kBlock, 0, st>>>(sink, iters, 0.9999f, 1e-3f);
      else k_fma_packed<<<grid, kBlock, 0, st>>>(sink, iters, 0.9999f, 1e-3f);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && r > 0 && ms < best[kind]) best[kind] = ms;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "ag_measure_fp32_peak");
  const double fma = (double)grid * kBlock * kChains * kRounds * iters;  // per launch
  out->scalar_ms = best[0];
  out->packed_ms = best[1];
  out->scalar_tflops = 2.0 * fma / (best[0] * 1e-3) / 1e12;
  out->packed_tflops = 4.0 * fma / (best[1] * 1e-3) / 1e12;
  out->grid = grid;
  out->block = kBlock;
  return AG_OK;
}

extern "C" ag_status ag_query_alu_peak(int device, ag_alu_peak* out) {
  if (!out) return agh::fail_invalid(nullptr, "ag_query_alu_peak: out is NULL");
  int sms = 0, khz = 0, major = 0, minor = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  if (e != cudaSuccess) return cuda_fail(e, "ag_query_alu_peak: device query");
  if (major < 6) return agh::fail_invalid(nullptr, "ag_query_alu_peak: compute capability below 6.0");
  // FP32 lanes per SM: half-rate FP32 parts (6.0, Volta/Turing 7.x, A100 8.0)
  // have 64, every later consumer and data-centre part (8.6+, 9.0, 10.x, 12.x) 128
  const bool lanes64 = (major == 6 && minor == 0) || major == 7 || (major == 8 && minor == 0);
  out->sm_count = (uint32_t)sms;
  out->fp32_lanes_per_sm = lanes64 ? 64u : 128u;
  out->max_sm_clock_khz = (uint32_t)khz;
  out->cc_major = (uint32_t)major;
  out->cc_minor = (uint32_t)minor;
  out->tflops = (double)sms * out->fp32_lanes_per_sm * 2.0 * (double)khz * 1e3 / 1e12;
  return AG_OK;
}

extern "C" ag_status ag_collision_tests_run(ag_ctx* ctx, uint64_t* tests) {
  ag_status s = agh::enter(ctx);
  if (s != AG_OK) return s;
  if (!tests) return agh::fail_invalid(ctx, "ag_collision_tests_run: tests is NULL");
  unsigned long long v = 0;
  s = agh::check_cuda(ctx, cudaMemcpyAsync(&v, ctx->fb.tests_run, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream),
                      "copy test count");
  if (s == AG_OK) s = agh::check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "synchronize");
  if (s == AG_OK) *tests = (uint64_t)v;
  return s;
}
