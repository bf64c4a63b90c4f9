// depth.cu — depth cameras by ray casting against the environments' boxes.
//
// The paper renders depth images through Isaac Gym's camera sensors (Sec. III,
// a graphics-API renderer) and names kernel-based ray casting as the way to
// render for many more robots (Sec. I, Sec. VII). Here every pixel is one
// thread: a pinhole camera mounted on the vehicle (offset o_b in the body
// frame, looking along body +x with body +z up) casts the ray
//   d = R (1, -(c + 0.5 - W/2) / f, -(r + 0.5 - H/2) / f),  f = (W/2) / tan(hfov/2)
// through pixel (r, c); the depth is the smallest t >= 0 at which the ray is
// inside a box (slab method in the box frame), which is the distance along
// the optical axis because d has a unit forward component; max_range when
// nothing is closer.
//
// One block renders 256 consecutive pixels of one camera. Its prologue turns
// each box into (R_b^T, camera origin in the box frame, half-extents) once in
// shared memory, so the per-pixel work is R_b^T d and three slabs per box.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "depth_internal.h"

namespace agk {
namespace {

constexpr int kDepthBlock = 256;
constexpr int kBoxRec = 15;  // R_b^T (9), camera origin in the box frame (3), half-extents (3)

__global__ void __launch_bounds__(kDepthBlock) k_render_depth(DepthArgs a) {
  extern __shared__ float sm[];  // [n_obs][kBoxRec]
  __shared__ float cam[12];      // R (9, row-major), origin (3)
  const uint32_t j = blockIdx.y;
  const uint32_t env = a.env_ids ? a.env_ids[j] : j;
  const uint32_t n = a.n;
  if (threadIdx.x == 0) {
    const float* st = a.state;
    Q4 q = {st[6 * n + env], st[7 * n + env], st[8 * n + env], st[9 * n + env]};
    normalize(q);
    float R[3][3];
    rotation(q, R);
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) cam[i * 3 + k] = R[i][k];
    for (int i = 0; i < 3; ++i)
      cam[9 + i] = st[i * n + env] + R[i][0] * a.offset[0] + R[i][1] * a.offset[1] + R[i][2] * a.offset[2];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < (int)a.n_obs; k += blockDim.x) {
    const float* bx = a.boxes + (size_t)k * 10 * n + env;
    float R[3][3];
    rotation(Q4{bx[6 * n], bx[7 * n], bx[8 * n], bx[9 * n]}, R);
    const V3 v = {cam[9] - bx[0], cam[10] - bx[n], cam[11] - bx[2 * n]};
    float* rec = sm + k * kBoxRec;
    for (int i = 0; i < 3; ++i)
      for (int m = 0; m < 3; ++m) rec[i * 3 + m] = R[m][i];  // R_b^T
    rec[9] = R[0][0] * v.x + R[1][0] * v.y + R[2][0] * v.z;
    rec[10] = R[0][1] * v.x + R[1][1] * v.y + R[2][1] * v.z;
    rec[11] = R[0][2] * v.x + R[1][2] * v.y + R[2][2] * v.z;
    rec[12] = bx[3 * n];
    rec[13] = bx[4 * n];
    rec[14] = bx[5 * n];
  }
  __syncthreads();
  const uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n_pix = a.width * a.height;
  if (pix >= n_pix) return;
  const uint32_t r = pix / a.width, c = pix - r * a.width;
  const float dy = -((float)c + 0.5f - 0.5f * (float)a.width) * a.inv_f;
  const float dz = -((float)r + 0.5f - 0.5f * (float)a.height) * a.inv_f;
  const V3 d = {cam[0] + cam[1] * dy + cam[2] * dz, cam[3] + cam[4] * dy + cam[5] * dz,
                cam[6] + cam[7] * dy + cam[8] * dz};
  float best = a.max_range;
  for (int k = 0; k < (int)a.n_obs; ++k) {
    const float* rec = sm + k * kBoxRec;
    float t_in = 0.f, t_out = best;  // only hits in [0, best) matter
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float di = rec[3 * i] * d.x + rec[3 * i + 1] * d.y + rec[3 * i + 2] * d.z;
      const float inv = __frcp_rn(di);
      const float t1 = (-rec[12 + i] - rec[9 + i]) * inv, t2 = (rec[12 + i] - rec[9 + i]) * inv;
      t_in = fmaxf(t_in, fminf(t1, t2));
      t_out = fminf(t_out, fmaxf(t1, t2));
    }
    if (t_in <= t_out) best = t_in;
  }
  a.out[(size_t)j * n_pix + pix] = best;
}

}  // namespace

cudaError_t launch_render_depth(const DepthArgs& a, cudaStream_t st) {
  const uint32_t n_pix = a.width * a.height;
  dim3 grid((n_pix + kDepthBlock - 1) / kDepthBlock, a.n_cams);
  const size_t smem = (size_t)a.n_obs * kBoxRec * sizeof(float);
  k_render_depth<<<grid, kDepthBlock, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace agk
