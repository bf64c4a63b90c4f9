// depth.cu — depth cameras by ray casting against the environments' boxes.
//
// The paper renders depth images through Isaac Gym's camera sensors (Sec. III,
// a graphics-API renderer) and names kernel-based ray casting as the way to
// render for many more robots (Sec. I, Sec. VII). Here every pixel's ray is
// traced on its own: a pinhole camera mounted on the vehicle (at a fixed
// offset in the body frame, looking along body +x with body +z up) casts the
// ray
//   d = R (1, -(c + 0.5 - W/2) / f, -(r + 0.5 - H/2) / f),  f = (W/2) / tan(hfov/2)
// through pixel (r, c); the depth is the smallest t >= 0 at which the ray is
// inside a box (slab method in the box frame), which is the distance along
// the optical axis because d has a unit forward component; max_range when
// nothing is closer.
//
// A block of 128 threads renders up to eight 32 x 32 tiles of one camera's
// image in turn, eight pixels per thread (column tx, rows ty, ty + 4, ...,
// ty + 28: each warp stores 32 consecutive pixels of a row). Once per block it
// turns each box into one 16-float record in shared memory: M = R_b^T R (the
// camera's axes in the box frame) and the slab bounds lo = -h - o_b,
// hi = h - o_b (o_b the camera origin in the box frame). Per pixel and box
// the ray's box-frame direction is then M (1, dy, dz) (six FMAs), followed by
// three reciprocals and the slab intervals; records are read as four
// broadcast 16-byte loads and reused for the thread's eight pixels.
//
// Once per block, warp w culls for the block's tiles w and w + 4,
// conservatively, the boxes that no ray of the tile can reach closer than
// max_range, and lists the live ones (ballot and popc), so the tile's loop
// visits only those. A
// box is culled when its bounding sphere (centre
// s in the camera frame, radius |h| with a rounding margin) lies beyond
// max_range along the axis, behind the camera, or outside one of the four
// planes through the camera origin that bound the tile's rays (y = dy x and
// z = dz x at the tile's extreme pixel centres). A culled box can change no
// pixel of the tile, so the image is the same as without culling. When each
// component of a live box's ray direction keeps one sign over the tile, the
// near and far slab bound of every axis is known for the whole tile, and the
// per-pixel min / max of the slab pairs is skipped (it would pick the same
// products).
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "ag.h"
#include "depth_internal.h"

namespace agk {
namespace {

constexpr int kDepthTile = 32;                           // tile edge in pixels
constexpr int kDepthThreads = 128;
constexpr int kDepthPix = kDepthTile * kDepthTile / kDepthThreads;  // pixels per thread: 8
constexpr int kDepthRows = kDepthThreads / kDepthTile;             // rows between a thread's pixels: 4
constexpr int kDepthTilesPerBlock = 8;                             // tiles of one camera per block

struct CamPose {
  float R[3][3];
  float o[3];
};

__device__ __forceinline__ CamPose camera_pose(const DepthArgs& a, uint32_t env) {
  const float* st = a.state;
  const uint32_t n = a.n;
  Q4 q = {st[6 * n + env], st[7 * n + env], st[8 * n + env], st[9 * n + env]};
  normalize(q);
  CamPose c;
  rotation(q, c.R);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    c.o[i] = st[i * n + env] + c.R[i][0] * a.offset[0] + c.R[i][1] * a.offset[1] + c.R[i][2] * a.offset[2];
  return c;
}

// record of box k: (M00 M01 M02 M10) (M11 M12 M20 M21) (M22 lo.x lo.y lo.z) (hi.x hi.y hi.z 0)
__device__ __forceinline__ void box_record(const DepthArgs& a, uint32_t env, const CamPose& c, int k, float4* rec) {
  const uint32_t n = a.n;
  const float* bx = a.boxes + (size_t)k * 10 * n + env;
  float Rb[3][3];
  rotation(Q4{bx[6 * n], bx[7 * n], bx[8 * n], bx[9 * n]}, Rb);
  const float v[3] = {c.o[0] - bx[0], c.o[1] - bx[n], c.o[2] - bx[2 * n]};
  float M[3][3], ob[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ob[i] = Rb[0][i] * v[0] + Rb[1][i] * v[1] + Rb[2][i] * v[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = Rb[0][i] * c.R[0][j] + Rb[1][i] * c.R[1][j] + Rb[2][i] * c.R[2][j];
  }
  const float h[3] = {bx[3 * n], bx[4 * n], bx[5 * n]};
  rec[0] = make_float4(M[0][0], M[0][1], M[0][2], M[1][0]);
  rec[1] = make_float4(M[1][1], M[1][2], M[2][0], M[2][1]);
  rec[2] = make_float4(M[2][2], -h[0] - ob[0], -h[1] - ob[1], -h[2] - ob[2]);
  rec[3] = make_float4(h[0] - ob[0], h[1] - ob[1], h[2] - ob[2], 0.f);
}

// Bounding sphere of box k in the camera frame: centre s, radius |h| with a
// rounding margin.
__device__ __forceinline__ float4 box_sphere(const DepthArgs& a, uint32_t env, const CamPose& c, int k) {
  const uint32_t n = a.n;
  const float* bx = a.boxes + (size_t)k * 10 * n + env;
  const float v[3] = {bx[0] - c.o[0], bx[n] - c.o[1], bx[2 * n] - c.o[2]};
  const float sx = c.R[0][0] * v[0] + c.R[1][0] * v[1] + c.R[2][0] * v[2];
  const float sy = c.R[0][1] * v[0] + c.R[1][1] * v[1] + c.R[2][1] * v[2];
  const float sz = c.R[0][2] * v[0] + c.R[1][2] * v[1] + c.R[2][2] * v[2];
  const float h0 = bx[3 * n], h1 = bx[4 * n], h2 = bx[5 * n];
  const float rho = 1.001f * sqrtf(h0 * h0 + h1 * h1 + h2 * h2) + 1e-4f * (fabsf(sx) + fabsf(sy) + fabsf(sz)) + 1e-6f;
  return make_float4(sx, sy, sz, rho);
}

// Rays of a tile: (1, y, z) in the camera frame with y in [ylo, yhi] and z in
// [zlo, zhi] (the tile's extreme pixel centres); ny_* = sqrt(1 + y^2) etc.
struct TileRays {
  float ylo, yhi, zlo, zhi, nylo, nyhi, nzlo, nzhi;
};

// The sphere cannot meet any ray of the tile at depth below max_range.
__device__ __forceinline__ bool sphere_culled(float4 s, const TileRays& t, float max_range) {
  const float rho = s.w;
  if (s.x - rho > max_range || s.x + rho < 0.f) return true;
  // signed distances to the four planes (positive inside the tile's pyramid)
  if (t.yhi * s.x - s.y < -rho * t.nyhi) return true;
  if (s.y - t.ylo * s.x < -rho * t.nylo) return true;
  if (t.zhi * s.x - s.z < -rho * t.nzhi) return true;
  if (s.z - t.zlo * s.x < -rho * t.nzlo) return true;
  return false;
}

// Flags of a live (tile, box) pair: kLive, and kFixedSigns when each
// component of the box-frame ray direction M (1, y, z) keeps one sign over
// the whole tile (it is linear in y and z, so the four corner rays decide,
// with a margin far above float32 rounding); then bit kNegX + i says that
// component i is negative, which fixes which slab bound is near and which is
// far for every pixel of the tile.
constexpr uint8_t kLive = 1, kFixedSigns = 2, kNegX = 2;

__device__ __forceinline__ uint8_t slab_signs(const float4* rec, const TileRays& t) {
  const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2];
  // rows (M_i0, M_i1, M_i2) of M
  const float m[3][3] = {{r0.x, r0.y, r0.z}, {r0.w, r1.x, r1.y}, {r1.z, r1.w, r2.x}};
  const float ys[2] = {t.ylo, t.yhi}, zs[2] = {t.zlo, t.zhi};
  uint8_t f = kLive | kFixedSigns;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    bool pos = true, neg = true;
    const float scale = fabsf(m[i][0]) + fmaxf(fabsf(t.ylo), fabsf(t.yhi)) * fabsf(m[i][1]) +
                        fmaxf(fabsf(t.zlo), fabsf(t.zhi)) * fabsf(m[i][2]);
    const float margin = 1e-5f * scale;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float d = m[i][0] + ys[c & 1] * m[i][1] + zs[c >> 1] * m[i][2];
      pos &= d > margin;
      neg &= d < -margin;
    }
    if (!pos && !neg) return kLive;          // the sign changes (or nearly) inside the tile
    if (neg) f |= (uint8_t)(1u << (kNegX + i));
  }
  return f;
}

// What a launch of k_render_depth does: render with fast reciprocals (the
// ray caster), render with correctly rounded reciprocals (to measure what the
// approximation moves), or only count the live (pixel, box) pairs.
enum DepthMode { kRenderFast = 0, kRenderIeee = 1, kCountLive = 2 };

template <int MODE>
__device__ __forceinline__ float depth_rcp(float x) {
  if (MODE == kRenderIeee) return 1.f / x;
  return __fdividef(1.f, x);
}

template <int MODE>
__global__ void __launch_bounds__(kDepthThreads) k_render_depth(DepthArgs a) {
  __shared__ float4 recs[AG_MAX_OBSTACLES * 4];
  __shared__ float4 spheres[AG_MAX_OBSTACLES];
  // per tile of the block: the live boxes (index, flags) in box order, and their number
  __shared__ uint8_t live_k[kDepthTilesPerBlock][AG_MAX_OBSTACLES];
  __shared__ uint8_t live_f[kDepthTilesPerBlock][AG_MAX_OBSTACLES];
  __shared__ int n_live[kDepthTilesPerBlock];
  __shared__ uint32_t tile_x0[kDepthTilesPerBlock], tile_y0[kDepthTilesPerBlock];  // pixel origin of each tile
  // block -> (camera, group of kDepthTilesPerBlock consecutive tiles); cameras cam0, cam0 + 1, ...
  const uint32_t tiles_x = (a.width + kDepthTile - 1) / kDepthTile;
  const uint32_t tiles = tiles_x * ((a.height + kDepthTile - 1) / kDepthTile);
  const uint32_t groups = (tiles + kDepthTilesPerBlock - 1) / kDepthTilesPerBlock;
  const uint32_t j = a.cam0 + blockIdx.x / groups;
  const uint32_t t_begin = (blockIdx.x % groups) * kDepthTilesPerBlock;
  const uint32_t t_end = min(t_begin + kDepthTilesPerBlock, tiles);
  const uint32_t env = a.env_ids ? a.env_ids[j] : j;
  // a camera id outside the fleet reads nothing and yields a NaN image
  const bool bad_env = env >= a.n;
  const uint32_t n_pix = a.width * a.height;
  const uint32_t tx = threadIdx.x & (kDepthTile - 1), ty = threadIdx.x / kDepthTile;
  const float half_w = 0.5f * (float)a.width, half_h = 0.5f * (float)a.height;
  const int n_obs = bad_env ? 0 : (int)a.n_obs;  // at most AG_MAX_OBSTACLES (checked when the context is created)
  // once per block: each box's record and its bounding sphere in the camera frame ...
  if ((int)threadIdx.x < n_obs) {
    const CamPose cam = camera_pose(a, env);
    for (int k = threadIdx.x; k < n_obs; k += kDepthThreads) {
      box_record(a, env, cam, k, recs + 4 * k);
      spheres[k] = box_sphere(a, env, cam, k);
    }
  }
  __syncthreads();
  // ... then warp w culls the boxes for tiles w, w + 4, ... of the block and lists the live ones
  constexpr uint32_t kWarps = kDepthThreads / 32;
  static_assert(kDepthTilesPerBlock % kWarps == 0, "whole tiles per warp");
  for (uint32_t w = threadIdx.x / 32; w < (uint32_t)kDepthTilesPerBlock; w += kWarps) {
    const uint32_t lane = threadIdx.x % 32, t = t_begin + w;
    if (t < t_end) {
      const uint32_t x0 = (t % tiles_x) * kDepthTile, y0 = (t / tiles_x) * kDepthTile;
      const uint32_t x1 = min(x0 + kDepthTile, a.width) - 1, y1 = min(y0 + kDepthTile, a.height) - 1;
      TileRays r;
      r.yhi = -((float)x0 + 0.5f - half_w) * a.inv_f;
      r.ylo = -((float)x1 + 0.5f - half_w) * a.inv_f;
      r.zhi = -((float)y0 + 0.5f - half_h) * a.inv_f;
      r.zlo = -((float)y1 + 0.5f - half_h) * a.inv_f;
      r.nyhi = sqrtf(1.f + r.yhi * r.yhi);
      r.nylo = sqrtf(1.f + r.ylo * r.ylo);
      r.nzhi = sqrtf(1.f + r.zhi * r.zhi);
      r.nzlo = sqrtf(1.f + r.zlo * r.zlo);
      int count = 0;
      for (int k0 = 0; k0 < n_obs; k0 += 32) {  // warp-uniform loop
        const int k = k0 + (int)lane;
        uint8_t f = 0;
        if (k < n_obs && !sphere_culled(spheres[k], r, a.max_range)) f = slab_signs(recs + 4 * k, r);
        const unsigned m = __ballot_sync(0xFFFFFFFFu, f != 0);
        if (f) {
          const int at = count + __popc(m & ((1u << lane) - 1u));
          live_k[w][at] = (uint8_t)k;
          live_f[w][at] = f;
        }
        count += __popc(m);
      }
      if (lane == 0) {
        n_live[w] = count;
        tile_x0[w] = x0;
        tile_y0[w] = y0;
      }
      if (MODE == kCountLive && lane == 0) {
        // pixels of tile t times its live boxes
        const unsigned long long px = (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
        atomicAdd(a.live_pairs, px * (unsigned long long)count);
      }
    }
  }
  if (MODE == kCountLive) return;
  __syncthreads();
  float* const out_cam = a.out + (size_t)j * n_pix;
  for (uint32_t t = t_begin; t < t_end; ++t) {
    const int tl = (int)(t - t_begin);
    const uint32_t x0 = tile_x0[tl], y0 = tile_y0[tl];
    const uint32_t col = x0 + tx;
    const float dy = -((float)col + 0.5f - half_w) * a.inv_f;
    float dz[kDepthPix], best[kDepthPix];
#pragma unroll
    for (int p = 0; p < kDepthPix; ++p) {
      dz[p] = -((float)(y0 + ty + p * kDepthRows) + 0.5f - half_h) * a.inv_f;
      best[p] = bad_env ? __int_as_float(0x7fc00000) : a.max_range;  // no box is tested for a bad id
    }
    for (int j = 0; j < n_live[tl]; ++j) {  // the same for the whole block
      const int k = live_k[tl][j];
      const uint8_t flags = live_f[tl][j];
      const float4 r0 = recs[4 * k], r1 = recs[4 * k + 1], r2 = recs[4 * k + 2], r3 = recs[4 * k + 3];
      // the column's part of M (1, dy, dz), shared by the thread's eight pixels
      const float cx = fmaf(dy, r0.y, r0.x), cy = fmaf(dy, r1.x, r0.w), cz = fmaf(dy, r1.w, r1.z);
      if (flags & kFixedSigns) {
        // slab bounds lo = (r2.y, r2.z, r2.w), hi = (r3.x, r3.y, r3.z): near is lo for a positive
        // direction component, hi for a negative one (the same min / max as below, known in advance)
        const bool nx = flags & (1u << kNegX), ny = flags & (2u << kNegX), nz = flags & (4u << kNegX);
        const float near_x = nx ? r3.x : r2.y, far_x = nx ? r2.y : r3.x;
        const float near_y = ny ? r3.y : r2.z, far_y = ny ? r2.z : r3.y;
        const float near_z = nz ? r3.z : r2.w, far_z = nz ? r2.w : r3.z;
#pragma unroll
        for (int p = 0; p < kDepthPix; ++p) {
          const float ix = depth_rcp<MODE>(fmaf(dz[p], r0.z, cx));
          const float iy = depth_rcp<MODE>(fmaf(dz[p], r1.y, cy));
          const float iz = depth_rcp<MODE>(fmaf(dz[p], r2.x, cz));
          const float t_in = fmaxf(fmaxf(0.f, near_x * ix), fmaxf(near_y * iy, near_z * iz));
          const float t_out = fminf(fminf(best[p], far_x * ix), fminf(far_y * iy, far_z * iz));
          if (t_in <= t_out) best[p] = t_in;
        }
        continue;
      }
#pragma unroll
      for (int p = 0; p < kDepthPix; ++p) {
        const float ix = depth_rcp<MODE>(fmaf(dz[p], r0.z, cx));
        const float iy = depth_rcp<MODE>(fmaf(dz[p], r1.y, cy));
        const float iz = depth_rcp<MODE>(fmaf(dz[p], r2.x, cz));
        const float ax = r2.y * ix, bx = r3.x * ix, ay = r2.z * iy, by = r3.y * iy, az = r2.w * iz, bz = r3.z * iz;
        // only hits in [0, best) matter
        const float t_in = fmaxf(fmaxf(0.f, fminf(ax, bx)), fmaxf(fminf(ay, by), fminf(az, bz)));
        const float t_out = fminf(fminf(best[p], fmaxf(ax, bx)), fminf(fmaxf(ay, by), fmaxf(az, bz)));
        if (t_in <= t_out) best[p] = t_in;
      }
    }
    if (col < a.width) {
#pragma unroll
      for (int p = 0; p < kDepthPix; ++p) {
        const uint32_t row = y0 + ty + p * kDepthRows;
        if (row < a.height) out_cam[(size_t)row * a.width + col] = best[p];
      }
    }
  }
}

}  // namespace

cudaError_t launch_render_depth(const DepthArgs& a_in, cudaStream_t st) {
  const uint64_t tiles = (uint64_t)((a_in.width + kDepthTile - 1) / kDepthTile) *
                         ((a_in.height + kDepthTile - 1) / kDepthTile);
  const uint64_t groups = (tiles + kDepthTilesPerBlock - 1) / kDepthTilesPerBlock;
  // at most 2^31 - 1 blocks per launch
  const uint64_t cams_per_launch = ((1ull << 31) - 1) / groups;
  DepthArgs a = a_in;
  for (uint64_t c0 = 0; c0 < a_in.n_cams; c0 += cams_per_launch) {
    const uint64_t nc = a_in.n_cams - c0 < cams_per_launch ? a_in.n_cams - c0 : cams_per_launch;
    a.cam0 = (uint32_t)c0;
    if (a.live_pairs) k_render_depth<kCountLive><<<(unsigned)(nc * groups), kDepthThreads, 0, st>>>(a);
    else if (a.ieee_div) k_render_depth<kRenderIeee><<<(unsigned)(nc * groups), kDepthThreads, 0, st>>>(a);
    else k_render_depth<kRenderFast><<<(unsigned)(nc * groups), kDepthThreads, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace agk
