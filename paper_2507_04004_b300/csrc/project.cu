// Projection, SH colour and tile culling of every (view, Gaussian), and the
// binning of kept (Gaussian, tile) pairs.
//
// arxiv 2507.04004, Sec. "3D Gaussian Splatting Representation":
//   mu_hat = R mu + t, d = e3^T mu_hat, mu' = pi_c(mu_hat / d),
//   Sigma' = J R Sigma R^T J^T (+ dilation), Sigma = R_g S S^T R_g^T,
//   colour from SH at the direction camera centre -> mean;
// Sec. "Fast Tile-based Culling": keep a tile iff the highest alpha the
// Gaussian reaches at one of its pixels is >= 1/255.  Sec. "Additional
// Strategies" (d): lanes carry a validity flag to one common exit and whole
// warps whose Gaussians are all cut stop early.
#include "gs_internal.h"

namespace gsb {

template <int DEG, bool BF16>
__global__ void __launch_bounds__(256) k_project(gs_map map, const gs_camera* __restrict__ cams, gs_config cfg,
                                                 Ws ws) {
  const int64_t n = ws.n;
  const int v = blockIdx.y;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = g < n;
  const int64_t e = (int64_t)v * n + g;
  const Cam cam = load_cam(cams, v);

  float mw[3] = {0.f, 0.f, 1.f};
  if (in_range) {
    mw[0] = map.mean[g];
    mw[1] = map.mean[n + g];
    mw[2] = map.mean[2 * n + g];
  }
  const float3 mh = to_camera(cam, mw[0], mw[1], mw[2]);
  bool ok = in_range && (mh.z > cfg.near_z);
  // Warp-level early stop: every lane of the warp is cut by the near plane.
  if (!__any_sync(kFull, ok)) {
    if (in_range) ws.rects[e] = empty_rect();
    return;
  }
  const float z = ok ? mh.z : 1.f;
  const float iz = 1.f / z;
  const float mx = __fmaf_rn(cam.fx * mh.x, iz, cam.cx);
  const float my = __fmaf_rn(cam.fy * mh.y, iz, cam.cy);
  // affine Jacobian of the projection with x/z, y/z clamped
  const float limx = cfg.fov_clamp * 0.5f * (float)ws.width / cam.fx;
  const float limy = cfg.fov_clamp * 0.5f * (float)ws.height / cam.fy;
  const float txc = fminf(limx, fmaxf(-limx, mh.x * iz));
  const float tyc = fminf(limy, fmaxf(-limy, mh.y * iz));
  const float j00 = cam.fx * iz, j02 = -cam.fx * txc * iz;
  const float j11 = cam.fy * iz, j12 = -cam.fy * tyc * iz;
  float m0[3], m1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    m0[j] = cam.R[j] * j00 + cam.R[6 + j] * j02;
    m1[j] = cam.R[3 + j] * j11 + cam.R[6 + j] * j12;
  }
  float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f, ls[3] = {0.f, 0.f, 0.f}, logit = 0.f;
  if (ok) {
    qw = map.quat[g]; qx = map.quat[n + g]; qy = map.quat[2 * n + g]; qz = map.quat[3 * n + g];
    ls[0] = map.log_scale[g]; ls[1] = map.log_scale[n + g]; ls[2] = map.log_scale[2 * n + g];
    logit = map.logit_opacity[g];
  }
  const float qq = qw * qw + qx * qx + qy * qy + qz * qz;
  ok = ok && qq > 0.f;
  const float qi = ok ? rsqrtf(qq) : 1.f;
  float Rg[3][3];
  quat_to_rot(qw * qi, qx * qi, qy * qi, qz * qi, Rg);
  // U = S R_g^T m0, V = S R_g^T m1; Sigma' = [[U.U, U.V], [U.V, V.V]] + dil I
  float U[3], Vv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float s = expf(ls[k]);
    U[k] = s * (Rg[0][k] * m0[0] + Rg[1][k] * m0[1] + Rg[2][k] * m0[2]);
    Vv[k] = s * (Rg[0][k] * m1[0] + Rg[1][k] * m1[1] + Rg[2][k] * m1[2]);
  }
  const float uu = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  const float vv = Vv[0] * Vv[0] + Vv[1] * Vv[1] + Vv[2] * Vv[2];
  const float uv = U[0] * Vv[0] + U[1] * Vv[1] + U[2] * Vv[2];
  const float dil = cfg.dilation;
  const float A = uu + dil, B = uv, C = vv + dil;
  // det Sigma' = |U x V|^2 + dil (|U|^2 + |V|^2) + dil^2 (no cancellation)
  const float cx0 = U[1] * Vv[2] - U[2] * Vv[1], cx1 = U[2] * Vv[0] - U[0] * Vv[2],
              cx2 = U[0] * Vv[1] - U[1] * Vv[0];
  const float det = cx0 * cx0 + cx1 * cx1 + cx2 * cx2 + dil * (uu + vv) + dil * dil;
  ok = ok && det > 0.f;
  const float idet = ok ? 1.f / det : 0.f;
  const float ca = C * idet, cb = -B * idet, cc = A * idet;
  const float o = 1.f / (1.f + expf(-logit));
  const float q_thr = 2.f * logf(o / cfg.alpha_min);
  ok = ok && q_thr > 0.f && ca > 0.f && cc > 0.f;

  // Tile box from the axis-aligned extent of the ellipse q <= q_thr
  // (|dx| <= sqrt(q_thr Sigma'_xx), |dy| <= sqrt(q_thr Sigma'_yy)), one pixel of slack.
  int tx0 = 1, ty0 = 0, tx1 = 0, ty1 = 0;
  if (ok) {
    const float hx = sqrtf(q_thr * A), hy = sqrtf(q_thr * C);
    const float Wf = (float)(ws.width - 1), Hf = (float)(ws.height - 1);
    const float px0 = floorf(mx - hx - 0.5f) - 1.f, px1 = ceilf(mx + hx - 0.5f) + 1.f;
    const float py0 = floorf(my - hy - 0.5f) - 1.f, py1 = ceilf(my + hy - 0.5f) + 1.f;
    if (px1 < 0.f || py1 < 0.f || px0 > Wf || py0 > Hf || !(px0 <= px1) || !(py0 <= py1)) {
      ok = false;
    } else {
      tx0 = (int)fmaxf(px0, 0.f) >> 4;
      tx1 = (int)fminf(px1, Wf) >> 4;
      ty0 = (int)fmaxf(py0, 0.f) >> 4;
      ty1 = (int)fminf(py1, Hf) >> 4;
    }
  }

  // View-dependent colour: dir = (mu - c_w) / |mu - c_w|.
  float rgb[3] = {0.f, 0.f, 0.f};
  if (ok) {
    const float3 cw = camera_centre(cam);
    float dx = mw[0] - cw.x, dy = mw[1] - cw.y, dz = mw[2] - cw.z;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[16];
    sh_basis<DEG>(dx, dy, dz, Y);
    constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) acc += sh_coeff<BF16>(map.sh_dc, map.sh_rest, n, g, k, ch) * Y[k];
      rgb[ch] = fmaxf(acc, 0.f);
    }
  }

  // Single exit: write the record and count kept tiles.
  uint32_t kept = 0;
  if (ok) {
    const float4 r0 = make_float4(mx, my, ca, cb);
    const float4 r1 = make_float4(cc, o, mh.z, q_thr);
    const Ellipse el = make_ellipse(r0, r1);
    uint32_t* cnt = ws.tile_count + (int64_t)v * ws.tiles_per_view;
    const int tiles_x = ws.tiles_x;
    for_each_kept_tile(el, tx0, ty0, tx1, ty1, ws.width, ws.height, [&](int tx, int ty) {
      atomicAdd(cnt + ty * tiles_x + tx, 1u);
      ++kept;
    });
    if (kept) {
      float4* rec = ws.records + 3 * e;
      rec[0] = r0;
      rec[1] = r1;
      rec[2] = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
      float4* adj = ws.adjoints + 3 * e;
      adj[0] = adj[1] = adj[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (in_range) ws.rects[e] = kept ? pack_rect(tx0, ty0, tx1, ty1) : empty_rect();
  // Append visible entries to the compact list, one atomic per warp.
  const unsigned vis = __ballot_sync(kFull, kept != 0);
  if (vis) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(vis) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ws.counters + kVisibleCount, (uint32_t)__popc(vis));
    base = __shfl_sync(kFull, base, leader);
    if (kept) ws.visible[base + __popc(vis & ((1u << lane) - 1u))] = (uint32_t)e;
  }
}

// One key per kept (Gaussian, tile) pair, written into the tile's bin:
// (depth key bits << 32) | Gaussian index.  The tile set is recomputed with
// the same function and the same stored floats as the count, so each bin
// receives exactly its counted number of keys.
__global__ void __launch_bounds__(256) k_emit(Ws ws) {
  if (ws.counters[kStatus] != 0) return;
  const uint32_t nvis = ws.counters[kVisibleCount];
  const int64_t n = ws.n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nvis; i += gridDim.x * blockDim.x) {
    const uint32_t e = ws.visible[i];
    const int v = (int)(e / (uint64_t)n);
    const uint32_t g = (uint32_t)(e - (uint64_t)v * n);
    const float4 r0 = ws.records[3 * (int64_t)e];
    const float4 r1 = ws.records[3 * (int64_t)e + 1];
    int tx0, ty0, tx1, ty1;
    unpack_rect(ws.rects[e], &tx0, &ty0, &tx1, &ty1);
    const Ellipse el = make_ellipse(r0, r1);
    const unsigned long long key = ((unsigned long long)__float_as_uint(r1.z) << 32) | g;
    const int64_t base = (int64_t)v * ws.tiles_per_view;
    const int tiles_x = ws.tiles_x;
    for_each_kept_tile(el, tx0, ty0, tx1, ty1, ws.width, ws.height, [&](int tx, int ty) {
      const int64_t t = base + ty * tiles_x + tx;
      const uint32_t pos = atomicAdd(ws.tile_cursor + t, 1u);
      if (pos < ws.tile_start[t] + ws.tile_count[t]) ws.keys[pos] = key;
      else atomicExch(ws.counters + kStatus, (uint32_t)GS_ERR_CUDA);
    });
  }
}

template <int DEG, bool BF16>
static cudaError_t launch_project_t(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                    cudaStream_t st) {
  dim3 grid((unsigned)((ws.n + 255) / 256), (unsigned)ws.views);
  trace_begin(kKProject, st);
  k_project<DEG, BF16><<<grid, 256, 0, st>>>(map, cams, cfg, ws);
  trace_end(st);
  return cudaGetLastError();
}

cudaError_t launch_project(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                           cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(ws.counters, 0, 16 * sizeof(uint32_t), st);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(ws.tile_count, 0, (size_t)ws.views * ws.tiles_per_view * sizeof(uint32_t), st);
  if (err != cudaSuccess) return err;
  const bool bf = map.sh_bf16 != 0;
  switch (map.sh_degree) {
    case 0: return bf ? launch_project_t<0, true>(map, cams, cfg, ws, st) : launch_project_t<0, false>(map, cams, cfg, ws, st);
    case 1: return bf ? launch_project_t<1, true>(map, cams, cfg, ws, st) : launch_project_t<1, false>(map, cams, cfg, ws, st);
    case 2: return bf ? launch_project_t<2, true>(map, cams, cfg, ws, st) : launch_project_t<2, false>(map, cams, cfg, ws, st);
    default: return bf ? launch_project_t<3, true>(map, cams, cfg, ws, st) : launch_project_t<3, false>(map, cams, cfg, ws, st);
  }
}

cudaError_t launch_emit(const Ws& ws, cudaStream_t st) {
  trace_begin(kKEmit, st);
  k_emit<<<sm_count() * 8, 256, 0, st>>>(ws);
  trace_end(st);
  return cudaGetLastError();
}

}  // namespace gsb
