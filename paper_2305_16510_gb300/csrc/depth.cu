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
// image in turn, eight pixels per thread: four consecutive columns of two
// rows 16 apart, so that each row's four depths leave as one 16-byte store
// (eight threads write a 128-byte row segment). Once per block it turns each
// box into one 16-float record in shared memory: M = R_b^T R (the camera's
// axes in the box frame) and the slab bounds lo = -h - o_b, hi = h - o_b
// (o_b the camera origin in the box frame). Per pixel and box the ray's
// box-frame direction is then M (1, dy, dz) (six FMAs, the column part
// shared by the thread's two rows), followed by three reciprocals and the
// slab intervals; records are read as four broadcast 16-byte loads and
// reused for the thread's eight pixels. Two pixels of a row travel as one
// FP32 pair, so the direction and slab products are packed FMAs / multiplies
// (__ffma2_rn, __fmul2_rn), each lane rounded as the scalar operation. A tile
// that no box reaches is only stored.
//
// Once per block, the warps cull for each of the block's tiles (a half
// warp per tile when there are at most 16 boxes), conservatively, the boxes
// that no ray of the tile can reach closer than max_range, and write the
// live ones' records, in box order, to the tile's list in shared memory
// (ballot and popc), so the tile's loop visits only those. A box is culled when its bounding sphere (centre s in the camera
// frame, radius |h| with a rounding margin) lies beyond max_range along the
// axis, behind the camera, or outside one of the four planes through the
// camera origin that bound the tile's rays (y = dy x and z = dz x at the
// tile's extreme pixel centres). A culled box can change no pixel of the
// tile, so the image is the same as without culling. When each component of
// a live box's ray direction keeps one sign over the tile, the near and far
// slab bound of every axis is known for the whole tile: the tile's copy of
// the record then holds them in place of lo and hi, and the per-pixel min /
// max of the slab pairs is skipped (it would pick the same products).
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "ag.h"
#include "depth_internal.h"

namespace agk {
namespace {

constexpr int kDepthTile = 32;                                      // tile edge in pixels
constexpr int kDepthThreads = 128;
constexpr int kDepthCols = 4;                                       // consecutive columns per thread
constexpr int kDepthColThreads = kDepthTile / kDepthCols;           // threads across a tile row: 8
constexpr int kDepthRowStep = kDepthThreads / kDepthColThreads;     // rows between a thread's rows: 16
constexpr int kDepthRowsPer = kDepthTile / kDepthRowStep;           // rows per thread: 2
constexpr int kDepthTilesPerBlock = 8;                              // tiles of one camera per block
static_assert(kDepthCols == 4 && kDepthRowsPer * kDepthRowStep == kDepthTile, "4 x 2 pixels per thread");

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
    c.o[i] = st[i * n + env] + fmaf(c.R[i][2], a.offset[2], fmaf(c.R[i][1], a.offset[1], c.R[i][0] * a.offset[0]));
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
    ob[i] = fmaf(Rb[2][i], v[2], fmaf(Rb[1][i], v[1], Rb[0][i] * v[0]));
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = fmaf(Rb[2][i], c.R[2][j], fmaf(Rb[1][i], c.R[1][j], Rb[0][i] * c.R[0][j]));
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
  const float sx = fmaf(c.R[2][0], v[2], fmaf(c.R[1][0], v[1], c.R[0][0] * v[0]));
  const float sy = fmaf(c.R[2][1], v[2], fmaf(c.R[1][1], v[1], c.R[0][1] * v[0]));
  const float sz = fmaf(c.R[2][2], v[2], fmaf(c.R[1][2], v[1], c.R[0][2] * v[0]));
  const float h0 = bx[3 * n], h1 = bx[4 * n], h2 = bx[5 * n];
  const float rho = 1.001f * sqrtf(h0 * h0 + h1 * h1 + h2 * h2) + 1e-4f * (fabsf(sx) + fabsf(sy) + fabsf(sz)) + 1e-6f;
  return make_float4(sx, sy, sz, rho);
}

// Rays of a tile: (1, y, z) in the camera frame with y in [ylo, yhi] and z in
// [zlo, zhi] (the tile's extreme pixel centres); ny_* = sqrt(1 + y^2) etc.
struct TileRays {
  float ylo, yhi, zlo, zhi, nylo, nyhi, nzlo, nzhi;
};

// sqrt(1 + y^2) as (1 + y^2) rsqrt(1 + y^2) with the hardware reciprocal square root.
__device__ __forceinline__ float norm1(float y) {
  const float q = fmaf(y, y, 1.f);
  return q * rsqrt_ftz(q);
}

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

// The fast reciprocal is the hardware approximation with subnormal inputs
// and results flushed to zero of the same sign (PTX rcp.approx.ftz.f32): a
// direction component below 2^-126 then acts as an exact 0, a ray parallel
// to that slab, as the slab test already handles.
template <int MODE>
__device__ __forceinline__ float depth_rcp(float x) {
  if (MODE == kRenderIeee) return 1.f / x;
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int MODE>
__device__ __forceinline__ float2 depth_rcp2(float2 x) {
  return make_float2(depth_rcp<MODE>(x.x), depth_rcp<MODE>(x.y));
}

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// The slab test of two pixels against one box: (ix, iy, iz) the reciprocals
// of their box-frame ray directions, (lo, hi) the slab bounds. With
// FIXED = true, lo holds each axis' near bound and hi its far bound for
// every pixel of the tile (a fixed sign of the direction component); else
// near and far are the min and max of the two products. Lowers best to the
// entry depth t_in where the ray meets the box at t_in in [0, best].
template <bool FIXED>
__device__ __forceinline__ void slab_pair(float2 ix, float2 iy, float2 iz, float lox, float loy, float loz, float hix,
                                          float hiy, float hiz, float& best0, float& best1) {
  const float2 ax = __fmul2_rn(dup2(lox), ix), bx = __fmul2_rn(dup2(hix), ix);
  const float2 ay = __fmul2_rn(dup2(loy), iy), by = __fmul2_rn(dup2(hiy), iy);
  const float2 az = __fmul2_rn(dup2(loz), iz), bz = __fmul2_rn(dup2(hiz), iz);
  float t_in0, t_out0, t_in1, t_out1;
  if (FIXED) {
    t_in0 = fmaxf(fmaxf(0.f, ax.x), fmaxf(ay.x, az.x));
    t_out0 = fminf(fminf(best0, bx.x), fminf(by.x, bz.x));
    t_in1 = fmaxf(fmaxf(0.f, ax.y), fmaxf(ay.y, az.y));
    t_out1 = fminf(fminf(best1, bx.y), fminf(by.y, bz.y));
  } else {
    t_in0 = fmaxf(fmaxf(0.f, fminf(ax.x, bx.x)), fmaxf(fminf(ay.x, by.x), fminf(az.x, bz.x)));
    t_out0 = fminf(fminf(best0, fmaxf(ax.x, bx.x)), fminf(fmaxf(ay.x, by.x), fmaxf(az.x, bz.x)));
    t_in1 = fmaxf(fmaxf(0.f, fminf(ax.y, bx.y)), fmaxf(fminf(ay.y, by.y), fminf(az.y, bz.y)));
    t_out1 = fminf(fminf(best1, fmaxf(ax.y, bx.y)), fminf(fmaxf(ay.y, by.y), fmaxf(az.y, bz.y)));
  }
  if (t_in0 <= t_out0) best0 = t_in0;
  if (t_in1 <= t_out1) best1 = t_in1;
}

template <int MODE>
__global__ void __launch_bounds__(kDepthThreads) k_render_depth(DepthArgs a) {
  __shared__ float4 recs[AG_MAX_OBSTACLES * 4];
  __shared__ float4 spheres[AG_MAX_OBSTACLES];
  // per tile of the block: the records of its live boxes in box order (n_obs slots of four float4,
  // dynamic shared memory), with near / far in place of lo / hi for a fixed-sign box, and their number
  extern __shared__ float4 tile_recs[];
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
  // this thread: columns cq .. cq + 3 and rows ry, ry + 16 of each tile
  const uint32_t cq = (threadIdx.x % kDepthColThreads) * kDepthCols, ry = threadIdx.x / kDepthColThreads;
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
  // ... then the warps cull the boxes for the block's tiles and list the live ones. A group of L lanes
  // takes one tile, its lane i boxes i, i + L, ...: L = 16 when the environment has at most 16 boxes
  // (two tiles per warp pass), else 32.
  constexpr uint32_t kWarps = kDepthThreads / 32;
  static_assert(kDepthTilesPerBlock % (2 * kWarps) == 0, "whole tiles per warp pass");
  const uint32_t L = n_obs <= 16 ? 16u : 32u;  // the same for the whole block
  const uint32_t lane = threadIdx.x % 32, g = lane / L, gl = lane % L;
  const unsigned gmask = L == 32u ? 0xFFFFFFFFu : (0xFFFFu << (16u * g));  // the ballot bits of this group
  for (uint32_t w0 = threadIdx.x / 32; w0 < (uint32_t)kDepthTilesPerBlock; w0 += kWarps * (32u / L)) {
    const uint32_t w = w0 + kWarps * g, t = t_begin + w;  // this group's tile
    const bool valid = t < t_end;
    const uint32_t tv = valid ? t : t_begin;               // an idle group computes on a real tile
    const uint32_t x0 = (tv % tiles_x) * kDepthTile, y0 = (tv / tiles_x) * kDepthTile;
    const uint32_t x1 = min(x0 + kDepthTile, a.width) - 1, y1 = min(y0 + kDepthTile, a.height) - 1;
    TileRays r;
    r.yhi = -((float)x0 + 0.5f - half_w) * a.inv_f;
    r.ylo = -((float)x1 + 0.5f - half_w) * a.inv_f;
    r.zhi = -((float)y0 + 0.5f - half_h) * a.inv_f;
    r.zlo = -((float)y1 + 0.5f - half_h) * a.inv_f;
    // the planes' normal lengths by the hardware square root (within a few ulp), far inside the
    // sphere radius' 1e-3 relative margin
    r.nyhi = norm1(r.yhi);
    r.nylo = norm1(r.ylo);
    r.nzhi = norm1(r.zhi);
    r.nzlo = norm1(r.zlo);
    int count = 0;
    for (int k0 = 0; k0 < n_obs; k0 += (int)L) {  // the same trip count for the whole warp
      const int k = k0 + (int)gl;
      uint8_t f = 0;
      if (valid && k < n_obs && !sphere_culled(spheres[k], r, a.max_range)) f = slab_signs(recs + 4 * k, r);
      const unsigned m = __ballot_sync(0xFFFFFFFFu, f != 0) & gmask;
      if (f && MODE != kCountLive) {
        const int at = count + __popc(m & ((1u << lane) - 1u));
        float4* const d = tile_recs + ((size_t)w * n_obs + at) * 4;
        const float4 q2 = recs[4 * k + 2], q3 = recs[4 * k + 3];
        float lo[3] = {q2.y, q2.z, q2.w}, hi[3] = {q3.x, q3.y, q3.z};
        if (f & kFixedSigns) {
#pragma unroll
          for (int i = 0; i < 3; ++i)
            if (f & (1u << (kNegX + i))) {  // negative component: the far bound is lo, the near one hi
              const float tmp = lo[i];
              lo[i] = hi[i];
              hi[i] = tmp;
            }
        }
        d[0] = recs[4 * k];
        d[1] = recs[4 * k + 1];
        d[2] = make_float4(q2.x, lo[0], lo[1], lo[2]);
        d[3] = make_float4(hi[0], hi[1], hi[2], (f & kFixedSigns) ? 1.f : 0.f);
      }
      count += __popc(m);
    }
    if (valid && gl == 0) {
      n_live[w] = count;
      tile_x0[w] = x0;
      tile_y0[w] = y0;
      if (MODE == kCountLive) {
        // pixels of tile t times its live boxes
        const unsigned long long px = (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
        atomicAdd(a.live_pairs, px * (unsigned long long)count);
      }
    }
  }
  if (MODE == kCountLive) return;
  __syncthreads();
  float* const out_cam = a.out + (size_t)j * n_pix;
  const float fill = bad_env ? __int_as_float(0x7fc00000) : a.max_range;  // no box is tested for a bad id
  for (uint32_t t = t_begin; t < t_end; ++t) {
    const int tl = (int)(t - t_begin);
    const uint32_t x0 = tile_x0[tl], y0 = tile_y0[tl];
    const uint32_t col0 = x0 + cq;
    const int nl = n_live[tl];  // the same for the whole block
    float best[kDepthRowsPer][kDepthCols];
#pragma unroll
    for (int r = 0; r < kDepthRowsPer; ++r)
#pragma unroll
      for (int c = 0; c < kDepthCols; ++c) best[r][c] = fill;
    if (nl > 0) {
      // ray (1, dy, dz) of each column and row; columns (cq, cq + 1) and (cq + 2, cq + 3) as pairs
      float2 dyp[2];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        dyp[h] = make_float2(-((float)(col0 + 2 * h) + 0.5f - half_w) * a.inv_f,
                             -((float)(col0 + 2 * h + 1) + 0.5f - half_w) * a.inv_f);
      float dz[kDepthRowsPer];
#pragma unroll
      for (int r = 0; r < kDepthRowsPer; ++r) dz[r] = -((float)(y0 + ry + r * kDepthRowStep) + 0.5f - half_h) * a.inv_f;
      const float4* const tr = tile_recs + (size_t)tl * n_obs * 4;
      for (int jl = 0; jl < nl; ++jl) {
        // (M00 M01 M02 M10) (M11 M12 M20 M21) (M22 lo) (hi fixed): lo / hi are near / far when fixed
        const float4 r0 = tr[4 * jl], r1 = tr[4 * jl + 1], r2 = tr[4 * jl + 2], r3 = tr[4 * jl + 3];
        // the column part of M (1, dy, dz), shared by the thread's two rows
        float2 cx[2], cy[2], cz[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cx[h] = __ffma2_rn(dyp[h], dup2(r0.y), dup2(r0.x));
          cy[h] = __ffma2_rn(dyp[h], dup2(r1.x), dup2(r0.w));
          cz[h] = __ffma2_rn(dyp[h], dup2(r1.w), dup2(r1.z));
        }
        const float2 mx = dup2(r0.z), my = dup2(r1.y), mz = dup2(r2.x);
        if (r3.w != 0.f) {
          // each axis' near and far bound known for the tile: the same min / max as below, in advance
#pragma unroll
          for (int r = 0; r < kDepthRowsPer; ++r) {
            const float2 z = dup2(dz[r]);
#pragma unroll
            for (int h = 0; h < 2; ++h)
              slab_pair<true>(depth_rcp2<MODE>(__ffma2_rn(z, mx, cx[h])), depth_rcp2<MODE>(__ffma2_rn(z, my, cy[h])),
                              depth_rcp2<MODE>(__ffma2_rn(z, mz, cz[h])), r2.y, r2.z, r2.w, r3.x, r3.y, r3.z,
                              best[r][2 * h], best[r][2 * h + 1]);
          }
          continue;
        }
#pragma unroll
        for (int r = 0; r < kDepthRowsPer; ++r) {
          const float2 z = dup2(dz[r]);
#pragma unroll
          for (int h = 0; h < 2; ++h)
            slab_pair<false>(depth_rcp2<MODE>(__ffma2_rn(z, mx, cx[h])), depth_rcp2<MODE>(__ffma2_rn(z, my, cy[h])),
                             depth_rcp2<MODE>(__ffma2_rn(z, mz, cz[h])), r2.y, r2.z, r2.w, r3.x, r3.y, r3.z,
                             best[r][2 * h], best[r][2 * h + 1]);
        }
      }
    }
    if (col0 < a.width) {
#pragma unroll
      for (int r = 0; r < kDepthRowsPer; ++r) {
        const uint32_t row = y0 + ry + r * kDepthRowStep;
        if (row >= a.height) continue;
        float* const o = out_cam + (size_t)row * a.width + col0;
        if (a.vec_store) {
          // width % 4 == 0 and a 16-byte aligned image: the four columns are inside and aligned
          *reinterpret_cast<float4*>(o) = make_float4(best[r][0], best[r][1], best[r][2], best[r][3]);
        } else {
#pragma unroll
          for (int c = 0; c < kDepthCols; ++c)
            if (col0 + c < a.width) o[c] = best[r][c];
        }
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
  // the tiles' live-box records: at most 8 x 64 x 64 B = 32 KB, within the default 48 KB per block
  const size_t smem = (size_t)kDepthTilesPerBlock * a_in.n_obs * 4 * sizeof(float4);
  DepthArgs a = a_in;
  a.vec_store = a.width % 4 == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
  for (uint64_t c0 = 0; c0 < a_in.n_cams; c0 += cams_per_launch) {
    const uint64_t nc = a_in.n_cams - c0 < cams_per_launch ? a_in.n_cams - c0 : cams_per_launch;
    a.cam0 = (uint32_t)c0;
    if (a.live_pairs) k_render_depth<kCountLive><<<(unsigned)(nc * groups), kDepthThreads, 0, st>>>(a);
    else if (a.ieee_div) k_render_depth<kRenderIeee><<<(unsigned)(nc * groups), kDepthThreads, smem, st>>>(a);
    else k_render_depth<kRenderFast><<<(unsigned)(nc * groups), kDepthThreads, smem, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace agk
