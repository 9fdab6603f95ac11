// Device-side building blocks shared by the rasterizer kernels (sm_103a).
//
// Everything here follows arxiv 2507.04004, Sec. "3D Gaussian Splatting
// Representation" (projection, Eq. alpha, SH colour) and Sec. "Fast
// Tile-based Culling"; constants that the paper takes from the 3DGS
// rasterizer it builds on arrive through gs_config.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gsb {

constexpr int kTile = 16;
constexpr int kTilePixels = kTile * kTile;
constexpr unsigned kFull = 0xffffffffu;

// Device view of the workspace parts (pointers resolved from gs_layout).
struct Ws {
  uint32_t* counters;     // [0] status [1] pairs needed [2] visible count [3] long-tile count
  float4* records;        // [V*N][3]
  uint2* rects;           // [V*N]
  float4* adjoints;       // [V*N][3]
  uint32_t* visible;      // [V*N]
  uint32_t* tile_count;   // [V*T]
  uint32_t* tile_start;   // [V*T]
  uint32_t* tile_cursor;  // [V*T]
  uint32_t* long_tiles;   // [V*T]
  unsigned long long* keys;      // [cap]
  unsigned long long* keys_alt;  // [cap]
  uint32_t* sorted_ids;   // [cap]
  float* view_stats;      // [V][4]
  int64_t n;
  int64_t cap;
  int32_t views, width, height, tiles_x, tiles_y, tiles_per_view;
};

enum CounterSlot { kStatus = 0, kPairsNeeded = 1, kVisibleCount = 2, kLongCount = 3 };

struct Cam {
  float R[9], t[3], fx, fy, cx, cy;
};

__device__ __forceinline__ Cam load_cam(const gs_camera* cams, int v) {
  Cam c;
  const gs_camera* p = cams + v;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = p->R[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) c.t[i] = p->t[i];
  c.fx = p->fx; c.fy = p->fy; c.cx = p->cx; c.cy = p->cy;
  return c;
}

// Camera-frame point R mu + t as explicit FMA chains; the z chain is the
// ordering depth key fmaf(R20, x, fmaf(R21, y, fmaf(R22, z, t2))).
__device__ __forceinline__ float3 to_camera(const Cam& c, float x, float y, float z) {
  float3 r;
  r.x = __fmaf_rn(c.R[0], x, __fmaf_rn(c.R[1], y, __fmaf_rn(c.R[2], z, c.t[0])));
  r.y = __fmaf_rn(c.R[3], x, __fmaf_rn(c.R[4], y, __fmaf_rn(c.R[5], z, c.t[1])));
  r.z = __fmaf_rn(c.R[6], x, __fmaf_rn(c.R[7], y, __fmaf_rn(c.R[8], z, c.t[2])));
  return r;
}

// Camera centre in the world, c_w = -R^T t.
__device__ __forceinline__ float3 camera_centre(const Cam& c) {
  return make_float3(-(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]),
                     -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]),
                     -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]));
}

// Rotation of a Gaussian from its normalised quaternion (w, x, y, z);
// Rg[i][j], column k is the k-th principal axis.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float Rg[3][3]) {
  Rg[0][0] = 1.f - 2.f * (y * y + z * z); Rg[0][1] = 2.f * (x * y - w * z); Rg[0][2] = 2.f * (x * z + w * y);
  Rg[1][0] = 2.f * (x * y + w * z); Rg[1][1] = 1.f - 2.f * (x * x + z * z); Rg[1][2] = 2.f * (y * z - w * x);
  Rg[2][0] = 2.f * (x * z - w * y); Rg[2][1] = 2.f * (y * z + w * x); Rg[2][2] = 1.f - 2.f * (x * x + y * y);
}

// Real spherical-harmonic basis, degree <= 3, at a unit direction, in
// Cartesian form with the Condon-Shortley phase; slot l*l + l + m.
// Normalisation constants: k0 = 1/(2 sqrt(pi)), k1 = sqrt(3/(4 pi)),
// k2a = sqrt(15/pi)/2, k2b = sqrt(5/pi)/4, k2c = sqrt(15/pi)/4,
// k3a = sqrt(35/(2 pi))/4, k3b = sqrt(105/pi)/2, k3c = sqrt(21/(2 pi))/4,
// k3d = sqrt(7/pi)/4, k3e = sqrt(105/pi)/4.
namespace shc {
constexpr float k0 = 0.28209479177387814f;
constexpr float k1 = 0.4886025119029199f;
constexpr float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
constexpr float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
constexpr float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
}  // namespace shc

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  using namespace shc;
  Y[0] = k0;
  if (DEG >= 1) { Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x; }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (3.f * zz - 1.f); Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -k3a * y * (3.f * xx - yy);
      Y[10] = k3b * x * y * z;
      Y[11] = -k3c * y * (5.f * zz - 1.f);
      Y[12] = k3d * z * (5.f * zz - 3.f);
      Y[13] = -k3c * x * (5.f * zz - 1.f);
      Y[14] = k3e * z * (xx - yy);
      Y[15] = -k3a * x * (xx - 3.f * yy);
    }
  }
}

// Gradient of each basis polynomial above w.r.t. (x, y, z) (the polynomials
// as functions on R^3; callers project out the radial part).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float3* dY) {
  using namespace shc;
  dY[0] = make_float3(0.f, 0.f, 0.f);
  if (DEG >= 1) {
    dY[1] = make_float3(0.f, -k1, 0.f);
    dY[2] = make_float3(0.f, 0.f, k1);
    dY[3] = make_float3(-k1, 0.f, 0.f);
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[4] = make_float3(k2a * y, k2a * x, 0.f);
    dY[5] = make_float3(0.f, -k2a * z, -k2a * y);
    dY[6] = make_float3(0.f, 0.f, 6.f * k2b * z);
    dY[7] = make_float3(-k2a * z, 0.f, -k2a * x);
    dY[8] = make_float3(2.f * k2c * x, -2.f * k2c * y, 0.f);
    if (DEG >= 3) {
      dY[9] = make_float3(-6.f * k3a * x * y, -k3a * (3.f * xx - 3.f * yy), 0.f);
      dY[10] = make_float3(k3b * y * z, k3b * x * z, k3b * x * y);
      dY[11] = make_float3(0.f, -k3c * (5.f * zz - 1.f), -10.f * k3c * y * z);
      dY[12] = make_float3(0.f, 0.f, k3d * (15.f * zz - 3.f));
      dY[13] = make_float3(-k3c * (5.f * zz - 1.f), 0.f, -10.f * k3c * x * z);
      dY[14] = make_float3(2.f * k3e * x * z, -2.f * k3e * y * z, k3e * (xx - yy));
      dY[15] = make_float3(-k3a * (3.f * xx - 3.f * yy), 6.f * k3a * x * y, 0.f);
    }
  }
}

// SH coefficient k of channel ch for Gaussian g (k = 0 is the DC array).
template <bool BF16>
__device__ __forceinline__ float sh_coeff(const void* dc, const void* rest, int64_t n, int64_t g, int k, int ch) {
  if (k == 0) {
    if (BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(dc)[ch * n + g]);
    return static_cast<const float*>(dc)[ch * n + g];
  }
  const int64_t off = ((int64_t)(k - 1) * 3 + ch) * n + g;
  if (BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(rest)[off]);
  return static_cast<const float*>(rest)[off];
}

// ----------------------------------------------------------------------------
// Per-pixel weight (Eq. alpha): the same FP32 expression is used by the
// forward, backward and Jacobian kernels so that their skip decisions agree.
struct AlphaEval {
  float alpha;  // min(alpha_max, o exp(power)), valid when pass
  float G;      // exp(power)
  float power;  // -q/2
  bool pass;    // alpha >= alpha_min
  bool clamped; // o exp(power) > alpha_max
};

__device__ __forceinline__ AlphaEval eval_alpha(float4 r0, float4 r1, float px, float py, float a_min,
                                                float a_max) {
  AlphaEval e;
  // explicit roundings: every kernel that includes this gets bit-identical alphas
  const float dx = __fsub_rn(px, r0.x), dy = __fsub_rn(py, r0.y);
  const float q2 = __fmaf_rn(__fmul_rn(r0.z, dx), dx, __fmul_rn(__fmul_rn(r1.x, dy), dy));
  e.power = __fmaf_rn(-0.5f, q2, -__fmul_rn(__fmul_rn(r0.w, dx), dy));
  e.G = __expf(e.power);
  const float a = __fmul_rn(r1.y, e.G);
  e.clamped = a > a_max;
  e.alpha = fminf(a_max, a);
  e.pass = (e.power <= 0.f) && (e.alpha >= a_min);
  return e;
}

// ----------------------------------------------------------------------------
// Tile culling (Sec. "Fast Tile-based Culling"): a tile is kept iff one of its
// pixel centres lies in the ellipse q <= q_thr, q_thr = 2 ln(o / alpha_min),
// i.e. the highest alpha the Gaussian reaches in the tile is >= alpha_min.
// Row by row the ellipse's chord gives the exact range of pixel centres
// inside it; the union of the chords' tile ranges over the 16 rows of a tile
// row is the kept set of that tile row.

struct Ellipse {
  float mx, my, a, b, c, q_thr, inv_a, det_c;
};

__device__ __forceinline__ Ellipse make_ellipse(float4 r0, float4 r1) {
  Ellipse e;
  e.mx = r0.x; e.my = r0.y; e.a = r0.z; e.b = r0.w; e.c = r1.x; e.q_thr = r1.w;
  // explicit round-to-nearest operations: the count and the emit kernels
  // must take bit-identical decisions
  e.inv_a = __fdiv_rn(1.f, e.a);
  e.det_c = __fsub_rn(__fmul_rn(e.a, e.c), __fmul_rn(e.b, e.b));
  return e;
}

// Tile-column range [*tl, *tr] of pixel centres inside the ellipse on pixel
// row y; false if the row holds none.
__device__ __forceinline__ bool row_tiles(const Ellipse& e, int y, int width, int* tl, int* tr) {
  const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), e.my);
  const float disc = __fsub_rn(__fmul_rn(e.a, e.q_thr), __fmul_rn(__fmul_rn(e.det_c, dy), dy));
  if (!(disc >= 0.f)) return false;
  const float half = __fmul_rn(__fsqrt_rn(disc), e.inv_a);
  const float xc = __fsub_rn(e.mx, __fmul_rn(__fmul_rn(e.b, dy), e.inv_a));
  const float xl = ceilf(__fsub_rn(__fsub_rn(xc, half), 0.5f));
  const float xr = floorf(__fsub_rn(__fadd_rn(xc, half), 0.5f));
  if (!(xl <= xr) || xr < 0.f || xl > (float)(width - 1)) return false;
  const int il = xl < 0.f ? 0 : (int)xl;
  const int ir = xr > (float)(width - 1) ? width - 1 : (int)xr;
  *tl = il >> 4;
  *tr = ir >> 4;
  return true;
}

// Calls f(tx, ty) for every kept tile inside the tile box, tile rows in
// ascending order, tiles ascending within a row.
template <class F>
__device__ __forceinline__ void for_each_kept_tile(const Ellipse& e, int tx0, int ty0, int tx1, int ty1, int width,
                                                   int height, F&& f) {
  for (int ty = ty0; ty <= ty1; ++ty) {
    const int y0 = ty * kTile, y1 = min(height - 1, y0 + kTile - 1);
    int lo = 1 << 30, hi = -1;
    bool gap = false;
    for (int y = y0; y <= y1; ++y) {
      int tl, tr;
      if (!row_tiles(e, y, width, &tl, &tr)) continue;
      if (hi >= 0 && (tl > hi + 1 || tr < lo - 1)) gap = true;
      lo = min(lo, tl);
      hi = max(hi, tr);
    }
    if (hi < 0) continue;
    lo = max(lo, tx0);
    hi = min(hi, tx1);
    if (!gap) {
      for (int tx = lo; tx <= hi; ++tx) f(tx, ty);
    } else {
      // rare: disjoint chords inside one tile row; test each tile exactly
      for (int tx = lo; tx <= hi; ++tx) {
        bool keep = false;
        for (int y = y0; y <= y1 && !keep; ++y) {
          int tl, tr;
          if (row_tiles(e, y, width, &tl, &tr)) keep = (tl <= tx && tx <= tr);
        }
        if (keep) f(tx, ty);
      }
    }
  }
}

__device__ __forceinline__ uint2 pack_rect(int x0, int y0, int x1, int y1) {
  return make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
}
__device__ __forceinline__ void unpack_rect(uint2 r, int* x0, int* y0, int* x1, int* y1) {
  *x0 = (int)(r.x & 0xffffu); *y0 = (int)(r.x >> 16); *x1 = (int)(r.y & 0xffffu); *y1 = (int)(r.y >> 16);
}
__device__ __forceinline__ bool rect_empty(uint2 r) { return (r.x & 0xffffu) > (r.y & 0xffffu); }

__device__ __forceinline__ uint2 empty_rect() { return make_uint2(1u, 0u); }

}  // namespace gsb
