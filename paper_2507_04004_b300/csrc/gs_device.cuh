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
// pixels per thread in the blend kernels (a tile is 256 / PPT threads)
constexpr int kFwdPPT = 4;
constexpr int kBwdPPT = 8;
constexpr int kWorkClasses = 64;  // classes of the blend backward's work list
static_assert(kWorkClasses % 32 == 0, "work classes are scanned 32 at a time");
constexpr int kBwdBatch = 128;  // Gaussians staged in shared memory per batch by the backward blend

// Passes of the binning's LSD radix sort of the visible entries: four on the
// 32-bit depth key, then one or two on the view (none for a single view).
__host__ __device__ inline int depth_sort_passes(int views) { return 4 + (views > 1 ? (views > 256 ? 2 : 1) : 0); }

// Device view of the workspace parts (pointers resolved from gs_layout).
struct Ws {
  uint32_t* counters;     // see CounterSlot
  float4* records;        // [V*N][3]
  uint2* rects;           // [V*N]
  float4* adjoints;       // [V*N][3]
  uint32_t* visible;      // [V*N] visible entries v*N + g, projection order
  uint32_t* vis_key;      // [V*N] depth key bits of each visible entry, projection order
  uint32_t* sort_key;     // [2][V*N] radix-sort buffers (keys)
  uint32_t* sort_val;     // [2][V*N] radix-sort buffers (entries)
  uint32_t* sorted;       // [V*N] visible entries in (view, depth key, index) order: the entry buffer of
                          // sort_val the sort's last pass leaves free (depth_sort_passes)
  uint32_t* radix_status; // [6][256] digit counts of the sort's passes, then [6][radix_tiles_max][256] tile status
  uint32_t* view_start;   // [V + 1] first sorted visible entry of each view
  uint32_t* gauss_list;   // [N] Gaussians visible in at least one view
  uint32_t* tile_count;   // [V*T]
  uint32_t* tile_start;   // [V*T]
  uint32_t* bucket_count;   // [V*tiles_y] row items per (view, tile row)
  uint32_t* bucket_start;   // [V*tiles_y]
  uint32_t* unit_first_e;   // [V + 1] first entry unit of each view
  uint32_t* unit_seg_e;     // [units_e_max] view of each entry unit
  uint32_t* unit_cnt_e;     // [units_e_max][tiles_y] row items per tile row of each entry unit, then offsets
  uint32_t* unit_first_r;   // [V*tiles_y + 1] first row unit of each bucket
  uint32_t* unit_seg_r;     // [units_r_max] bucket of each row unit
  uint32_t* unit_cnt_r;     // [units_r_max][tiles_x] pairs per tile of each row unit, then offsets
  uint32_t* row_items;      // [cap] entry of each row item, by bucket, (depth key, index) order inside
  uint32_t* row_span;       // [cap] packed kept-tile span of each row item
  uint32_t* sorted_ids;   // [cap]
  float* view_stats;      // [V][4]
  uint32_t* work_fill;    // [kWorkClasses] items per work class
  uint32_t* work_lists;   // [kWorkClasses][V*T] (view, tile) items of each class
  int64_t n;
  int64_t cap;
  int64_t units_e_max, units_r_max, radix_tiles_max;
  int32_t views, width, height, tiles_x, tiles_y, tiles_per_view;
};

// Binning granularity: an entry unit is a run of consecutive sorted visible
// entries of one view, a row unit a run of row items of one (view, tile row)
// bucket; one warp processes one unit.  Inputs come in depth order, nearest
// (largest on screen, most rows and tiles) first, so unit sizes grow
// geometrically along a segment - kUnitFirst, 2 kUnitFirst, ... up to the
// cap (kEntryUnit, kRowUnit) - which splits the heavy front finely.
constexpr int kEntryUnit = 256;
constexpr int kRowUnit = 128;
constexpr int kUnitFirst = 4;

// Units of the growing schedule before the cap is reached, and the items they hold.
__host__ __device__ constexpr int unit_ramp(int cap) { return cap <= kUnitFirst ? 0 : 1 + unit_ramp(cap / 2); }
// First item of unit k of a segment (units of kUnitFirst * 2^k items, then `cap`).
__host__ __device__ inline int64_t unit_start(int64_t k, int cap) {
  const int r = unit_ramp(cap);
  if (k <= r) return (int64_t)kUnitFirst * ((int64_t(1) << k) - 1);
  return (int64_t)kUnitFirst * ((int64_t(1) << r) - 1) + (k - r) * cap;
}
// Units covering c items.
__host__ __device__ inline uint32_t unit_count(uint32_t c, int cap) {
  const int r = unit_ramp(cap);
  const int64_t ramp_items = (int64_t)kUnitFirst * ((int64_t(1) << r) - 1);
  if (c == 0) return 0;
  if ((int64_t)c <= ramp_items) {
    uint32_t k = 0;
    while (unit_start(k + 1, cap) < (int64_t)c) ++k;
    return k + 1;
  }
  return (uint32_t)(r + (c - ramp_items + cap - 1) / cap);
}
// Entries per tile of the sort's passes (256 threads x 8).
constexpr int kRadixTileEntries = 2048;

enum CounterSlot {
  kStatus = 0, kPairsNeeded = 1, kVisibleCount = 2, kEntryUnits = 3, kRowCount = 4, kGaussCount = 5, kRowUnits = 6,
  kRadixTicket = 8,  // [8, 14): tile tickets of the sort's passes
  kProjectTicket = 15  // chunk tickets of the projection
};

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

// sum_k w[k] grad Y_k(x, y, z) for the polynomials above, without forming
// the per-k gradients as an array.
template <int DEG>
__device__ __forceinline__ float3 sh_weighted_grad(const float* w, float x, float y, float z) {
  using namespace shc;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (DEG >= 1) {
    gy -= k1 * w[1];
    gz += k1 * w[2];
    gx -= k1 * w[3];
  }
  if (DEG >= 2) {
    gx += k2a * y * w[4]; gy += k2a * x * w[4];
    gy -= k2a * z * w[5]; gz -= k2a * y * w[5];
    gz += 6.f * k2b * z * w[6];
    gx -= k2a * z * w[7]; gz -= k2a * x * w[7];
    gx += 2.f * k2c * x * w[8]; gy -= 2.f * k2c * y * w[8];
    if (DEG >= 3) {
      const float xx = x * x, yy = y * y, zz = z * z;
      gx -= 6.f * k3a * x * y * w[9]; gy -= k3a * (3.f * xx - 3.f * yy) * w[9];
      gx += k3b * y * z * w[10]; gy += k3b * x * z * w[10]; gz += k3b * x * y * w[10];
      gy -= k3c * (5.f * zz - 1.f) * w[11]; gz -= 10.f * k3c * y * z * w[11];
      gz += k3d * (15.f * zz - 3.f) * w[12];
      gx -= k3c * (5.f * zz - 1.f) * w[13]; gz -= 10.f * k3c * x * z * w[13];
      gx += 2.f * k3e * x * z * w[14]; gy -= 2.f * k3e * y * z * w[14]; gz += k3e * (xx - yy) * w[14];
      gx -= k3a * (3.f * xx - 3.f * yy) * w[15]; gy += 6.f * k3a * x * y * w[15];
    }
  }
  return make_float3(gx, gy, gz);
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
// Blend-kernel form of a projected Gaussian (Eq. alpha in the log2 domain):
//   p2(px, py) = ha dx^2 + hb dx dy + hc dy^2 + log2(o),  dx = px - mx,
//   ha = -a log2(e) / 2, hb = -b log2(e), hc = -c log2(e) / 2,
// so o exp(-q/2) = 2^p2 and the alpha_min test is p2 >= log2(alpha_min),
// taken before any exponential.  The forward, backward and Jacobian kernels
// stage records through stage_gaussian() and evaluate p2 with blend_p2(),
// both with explicit roundings, so their decisions are bit-identical.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

struct Staged {
  float4 g0;  // mx, my, ha, hb
  float4 g1;  // hc, log2(o), depth, 1/o
};

__device__ __forceinline__ Staged stage_gaussian(float4 r0, float4 r1) {
  Staged s;
  s.g0 = make_float4(r0.x, r0.y, __fmul_rn(-0.5f * kLog2e, r0.z), __fmul_rn(-kLog2e, r0.w));
  s.g1 = make_float4(__fmul_rn(-0.5f * kLog2e, r1.x), __log2f(r1.y), r1.z, __frcp_rn(r1.y));
  return s;
}

// p2 = dy (hc dy + hb dx) + (ha dx^2 + log2 o): the bracketed terms depend on
// the pixel column only, so a thread that owns a column of pixels forms them
// once (col_terms) and pays three operations per pixel (col_p2).
struct ColTerms {
  float A;   // ha dx^2 + log2 o
  float B;   // hb dx
  float hc;
  float my;
};

__device__ __forceinline__ ColTerms col_terms(float4 g0, float4 g1, float px) {
  const float dx = __fsub_rn(px, g0.x);
  return ColTerms{__fmaf_rn(__fmul_rn(g0.z, dx), dx, g1.y), __fmul_rn(g0.w, dx), g1.x, g0.y};
}

__device__ __forceinline__ float col_p2(const ColTerms& c, float py) {
  const float dy = __fsub_rn(py, c.my);
  return __fmaf_rn(dy, __fmaf_rn(c.hc, dy, c.B), c.A);
}

__device__ __forceinline__ float blend_p2(float4 g0, float4 g1, float px, float py) {
  return col_p2(col_terms(g0, g1, px), py);
}

// 2^x on the special-function unit (PTX ex2.approx.ftz.f32: relative error
// near 2^-22, subnormal results flushed to zero).  Every alpha that takes
// part in compositing is >= alpha_min, far from the subnormal range; the
// forward, backward and Jacobian kernels all use this one function, so they
// see the same alpha.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / x on the special-function unit (PTX rcp.approx.ftz.f32, relative
// error near 2^-23).  The backward kernels divide only by 1 - alpha, which
// lies in [1 - alpha_max, 1], so no range handling is needed around it.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Four-float reduction into global memory with no value returned (PTX
// red.global.add.v4.f32): unlike an atomic whose result registers must be
// written back before they are reused, nothing in the issuing warp waits for it.
__device__ __forceinline__ void red_add4(float4* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

// Asynchronous 4-byte global -> shared copies (cp.async), their commit and
// the wait for all of a thread's outstanding copies.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Packed FP32 pairs: the blend kernels evaluate two vertically adjacent
// pixels per instruction with the sm_100+ f32x2 FMA/ADD/MUL.  Each half is
// rounded exactly like the scalar __fmaf_rn / __fadd_rn / __fmul_rn, so
// col_p2x2 returns the bits col_p2 returns for each pixel.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 col_p2x2(const ColTerms& c, float2 py) {
  const float2 dy = __fadd2_rn(py, f2(-c.my));
  return __ffma2_rn(dy, __ffma2_rn(f2(c.hc), dy, f2(c.B)), f2(c.A));
}

// ----------------------------------------------------------------------------
// Tile culling (Sec. "Fast Tile-based Culling"): a tile is kept iff one of its
// pixel centres lies in the ellipse q <= q_thr, q_thr = 2 ln(o / alpha_min),
// i.e. the highest alpha the Gaussian reaches in the tile is >= alpha_min.
// Row by row the ellipse's chord gives the exact range of pixel centres
// inside it; the union of the chords' tile ranges over the 16 rows of a tile
// row is the kept set of that tile row.

// Per-ellipse constants of the chord computation: with dy = y + 0.5 - my,
//   disc = a q_thr - det dy^2,  det = a c - b^2,
//   chord centre - 0.5 = (mx - 0.5) - (b / a) dy,  half width = sqrt(disc) / a.
struct Ellipse {
  float my, aq, det, inv_a, b_a, mxm;
};

__device__ __forceinline__ Ellipse make_ellipse(float4 r0, float4 r1) {
  Ellipse e;
  // explicit roundings and single-instruction approximations (no branches):
  // every kernel that evaluates a chord takes bit-identical decisions
  const float a = r0.z, b = r0.w, c = r1.x;
  e.my = r0.y;
  e.inv_a = __fdividef(1.f, a);
  e.det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
  e.aq = __fmul_rn(a, r1.w);
  e.b_a = __fmul_rn(b, e.inv_a);
  e.mxm = __fsub_rn(r0.x, 0.5f);
  return e;
}

// Pixel-centre columns [xl, xr] inside the ellipse on two pixel rows, whose
// centres are yc.x and yc.y (y + 0.5), clamped to the image; ok[k] is false
// if row k holds none.  The arithmetic runs on packed FP32 pairs, each half
// rounded exactly as row_tiles rounds it, so both take the same decisions.
// Written without branches so that the lanes of a warp stay converged across
// the 16 rows of a tile row.
__device__ __forceinline__ void row_px2(const Ellipse& e, float2 yc, float wm1, float2* xl, float2* xr, bool ok[2]) {
  const float2 dy = __fadd2_rn(yc, make_float2(-e.my, -e.my));
  const float2 disc = __ffma2_rn(__fmul2_rn(make_float2(-e.det, -e.det), dy), dy, make_float2(e.aq, e.aq));
  const float2 dpos = make_float2(fmaxf(disc.x, 1e-30f), fmaxf(disc.y, 1e-30f));
  const float2 half = __fmul2_rn(__fmul2_rn(dpos, make_float2(rsqrtf(dpos.x), rsqrtf(dpos.y))),
                                 make_float2(e.inv_a, e.inv_a));
  const float2 cm = __ffma2_rn(make_float2(-e.b_a, -e.b_a), dy, make_float2(e.mxm, e.mxm));
  const float2 a = __fadd2_rn(cm, make_float2(-half.x, -half.y)), b = __fadd2_rn(cm, half);
  const float l0 = ceilf(a.x), l1 = ceilf(a.y), r0 = floorf(b.x), r1 = floorf(b.y);
  *xl = make_float2(fminf(fmaxf(l0, 0.f), wm1), fminf(fmaxf(l1, 0.f), wm1));
  *xr = make_float2(fminf(fmaxf(r0, 0.f), wm1), fminf(fmaxf(r1, 0.f), wm1));
  ok[0] = (disc.x >= 0.f) & (l0 <= r0) & (r0 >= 0.f) & (l0 <= wm1);
  ok[1] = (disc.y >= 0.f) & (l1 <= r1) & (r1 >= 0.f) & (l1 <= wm1);
}

// Tile-column range [*tl, *tr] of pixel centres inside the ellipse on pixel
// row y; false if the row holds none (the per-tile test of tile_kept()).
__device__ __forceinline__ bool row_tiles(const Ellipse& e, int y, int width, int* tl, int* tr) {
  const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), e.my);
  const float disc = __fmaf_rn(-__fmul_rn(e.det, dy), dy, e.aq);
  const float dpos = fmaxf(disc, 1e-30f);
  const float half = __fmul_rn(__fmul_rn(dpos, rsqrtf(dpos)), e.inv_a);  // sqrt(disc) / a
  const float cm = __fmaf_rn(-e.b_a, dy, e.mxm);                         // chord centre - 0.5
  const float wm1 = (float)(width - 1);
  const float xl = ceilf(__fsub_rn(cm, half));
  const float xr = floorf(__fadd_rn(cm, half));
  const bool ok = (disc >= 0.f) & (xl <= xr) & (xr >= 0.f) & (xl <= wm1);
  *tl = (int)fminf(fmaxf(xl, 0.f), wm1) >> 4;
  *tr = (int)fminf(fmaxf(xr, 0.f), wm1) >> 4;
  return ok;
}

// Kept tiles of tile row ty: the columns [lo, hi] hull the 16 chords' tile
// ranges.  The hull is kept in pixels; gap is set when a chord lies more
// than 16 pixels beyond the hull of the rows before it, the only way the
// chords' tile ranges can leave a tile between them (rare: very thin tilted
// ellipses).  A span with gap set is conservative: only the tiles that
// tile_kept() confirms belong to the set.
struct RowSpan {
  int lo, hi;
  bool gap;
};

__device__ __forceinline__ RowSpan row_span(const Ellipse& e, int ty, int width, int height) {
  const int y0 = ty * kTile, y1 = min(height - 1, y0 + kTile - 1);
  const float wm1 = (float)(width - 1);
  float lo = 3.0e38f, hi = -1.f;  // hull of the rows' clamped pixel ranges
  bool gap = false;
  const float yc = (float)y0 + 0.5f;  // row centre, exact for any image row
#pragma unroll
  for (int r = 0; r < kTile; r += 2) {
    float2 xl, xr;
    bool ok[2];
    row_px2(e, make_float2(yc + (float)r, yc + (float)(r + 1)), wm1, &xl, &xr, ok);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float l = k ? xl.y : xl.x, rr = k ? xr.y : xr.x;
      const bool o = ok[k] & (y0 + r + k <= y1);
      gap |= o & (hi >= 0.f) & ((l > hi + 16.f) | (rr < lo - 16.f));
      lo = o ? fminf(lo, l) : lo;
      hi = o ? fmaxf(hi, rr) : hi;
    }
  }
  RowSpan s{1 << 30, -1, gap};
  if (hi >= 0.f) {
    s.lo = (int)lo >> 4;
    s.hi = (int)hi >> 4;
  }
  return s;
}

// Exact test of one tile of a gap row: one of its pixel rows' chords reaches it.
__device__ __forceinline__ bool tile_kept(const Ellipse& e, int tx, int ty, int width, int height) {
  const int y0 = ty * kTile, y1 = min(height - 1, y0 + kTile - 1);
  for (int y = y0; y <= y1; ++y) {
    int tl, tr;
    if (row_tiles(e, y, width, &tl, &tr) && tl <= tx && tx <= tr) return true;
  }
  return false;
}

// Packed span of a row item: lo | hi << 12 | gap << 31 (lo > hi: empty).
__device__ __forceinline__ uint32_t pack_span(const RowSpan& s) {
  if (s.hi < 0) return 0xfffu;
  return (uint32_t)s.lo | ((uint32_t)s.hi << 12) | (s.gap ? 0x80000000u : 0u);
}
__device__ __forceinline__ RowSpan unpack_span(uint32_t p) {
  RowSpan s;
  s.lo = (int)(p & 0xfffu);
  s.hi = (int)((p >> 12) & 0xfffu);
  s.gap = (p >> 31) != 0;
  return s;
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
