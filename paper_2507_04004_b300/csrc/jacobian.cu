// Pose Jacobian rows for tracking (arxiv 2507.04004, Eq. 3dgs_jacobi and the
// manifold derivative after it; camera factor option 2 of Sec. "Camera Factor
// (Option 2)"): for each selected pixel, dC/dxi (3x6) under the right
// perturbation T Exp(xi), xi = (rho, theta).  Forward mode: per contributing
// Gaussian, the six tangents of (mu', conic, colour) -- including the
// high-order SH term through the viewing direction -- and, along the pixel's
// front-to-back list, the carried sum S = sum_{j<i} dalpha_j / (1 - alpha_j)
// that gives dT_i = -T_i S.
#include "gs_internal.h"

namespace gsb {

struct Tangents {
  float mx[6], my[6], a[6], b[6], c[6], col[3][6];
};

template <int DEG, bool BF16>
__device__ void pose_tangents(const gs_map& map, int64_t g, const Cam& cam, const gs_config& cfg, int width,
                              int height, float4 R0, float4 R1, Tangents& tg) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const int64_t n = map.n;
  const float mu[3] = {map.mean[g], map.mean[n + g], map.mean[2 * n + g]};
  float q[4] = {map.quat[g], map.quat[n + g], map.quat[2 * n + g], map.quat[3 * n + g]};
  const float qi = rsqrtf(fmaxf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3], 1e-30f));
  float Rg[3][3];
  quat_to_rot(q[0] * qi, q[1] * qi, q[2] * qi, q[3] * qi, Rg);
  float s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = expf(map.log_scale[k * n + g]);
  const float3 mh = to_camera(cam, mu[0], mu[1], mu[2]);
  const float iz = 1.f / mh.z, iz2 = iz * iz;
  const float limx = cfg.fov_clamp * 0.5f * (float)width / cam.fx;
  const float limy = cfg.fov_clamp * 0.5f * (float)height / cam.fy;
  const float txr = mh.x * iz, tyr = mh.y * iz;
  const bool clx = txr > limx || txr < -limx, cly = tyr > limy || tyr < -limy;
  const float txc = fminf(limx, fmaxf(-limx, txr)), tyc = fminf(limy, fmaxf(-limy, tyr));
  const float j00 = cam.fx * iz, j02 = -cam.fx * txc * iz, j11 = cam.fy * iz, j12 = -cam.fy * tyc * iz;
  float m0[3], m1[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    m0[j] = cam.R[j] * j00 + cam.R[6 + j] * j02;
    m1[j] = cam.R[3 + j] * j11 + cam.R[6 + j] * j12;
  }
  float U[3], Vv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[k] = s[k] * (Rg[0][k] * m0[0] + Rg[1][k] * m0[1] + Rg[2][k] * m0[2]);
    Vv[k] = s[k] * (Rg[0][k] * m1[0] + Rg[1][k] * m1[1] + Rg[2][k] * m1[2]);
  }
  const float qa = R0.z, qb = R0.w, qc = R1.x;
  const float3 cw = camera_centre(cam);
  const float c_w[3] = {cw.x, cw.y, cw.z};
  float dv[3] = {mu[0] - cw.x, mu[1] - cw.y, mu[2] - cw.z};
  const float inv = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const float dir[3] = {dv[0] * inv, dv[1] * inv, dv[2] * inv};
  float Y[16];
  float3 dY[16];
  sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
  sh_basis_grad<DEG>(dir[0], dir[1], dir[2], dY);
  float3 Gd[3];
  bool on[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float raw = 0.5f;
    float3 gd = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float c = sh_coeff<BF16>(map.sh_dc, map.sh_rest, n, g, k, ch);
      raw += c * Y[k];
      gd.x += c * dY[k].x; gd.y += c * dY[k].y; gd.z += c * dY[k].z;
    }
    Gd[ch] = gd;
    on[ch] = raw > 0.f;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float dmh[3], dcw[3], rot0[3] = {0.f, 0.f, 0.f}, rot1[3] = {0.f, 0.f, 0.f};
    if (k < 3) {
#pragma unroll
      for (int i = 0; i < 3; ++i) { dmh[i] = cam.R[3 * i + k]; dcw[i] = (i == k) ? -1.f : 0.f; }
    } else {
      const int j = k - 3;
      // e_j x mu, c_w x e_j, m x e_j
      float exm[3], cxe[3];
      exm[0] = (j == 1) ? mu[2] : (j == 2) ? -mu[1] : 0.f;
      exm[1] = (j == 2) ? mu[0] : (j == 0) ? -mu[2] : 0.f;
      exm[2] = (j == 0) ? mu[1] : (j == 1) ? -mu[0] : 0.f;
      cxe[0] = (j == 2) ? c_w[1] : (j == 1) ? -c_w[2] : 0.f;
      cxe[1] = (j == 0) ? c_w[2] : (j == 2) ? -c_w[0] : 0.f;
      cxe[2] = (j == 1) ? c_w[0] : (j == 0) ? -c_w[1] : 0.f;
      rot0[0] = (j == 2) ? m0[1] : (j == 1) ? -m0[2] : 0.f;
      rot0[1] = (j == 0) ? m0[2] : (j == 2) ? -m0[0] : 0.f;
      rot0[2] = (j == 1) ? m0[0] : (j == 0) ? -m0[1] : 0.f;
      rot1[0] = (j == 2) ? m1[1] : (j == 1) ? -m1[2] : 0.f;
      rot1[1] = (j == 0) ? m1[2] : (j == 2) ? -m1[0] : 0.f;
      rot1[2] = (j == 1) ? m1[0] : (j == 0) ? -m1[1] : 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dmh[i] = cam.R[3 * i] * exm[0] + cam.R[3 * i + 1] * exm[1] + cam.R[3 * i + 2] * exm[2];
        dcw[i] = cxe[i];
      }
    }
    tg.mx[k] = cam.fx * (dmh[0] * iz - mh.x * dmh[2] * iz2);
    tg.my[k] = cam.fy * (dmh[1] * iz - mh.y * dmh[2] * iz2);
    const float dj00 = -cam.fx * dmh[2] * iz2, dj11 = -cam.fy * dmh[2] * iz2;
    const float dj02 = clx ? cam.fx * txc * dmh[2] * iz2 : -cam.fx * dmh[0] * iz2 + 2.f * cam.fx * txc * dmh[2] * iz2;
    const float dj12 = cly ? cam.fy * tyc * dmh[2] * iz2 : -cam.fy * dmh[1] * iz2 + 2.f * cam.fy * tyc * dmh[2] * iz2;
    float dm0[3], dm1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dm0[j] = cam.R[j] * dj00 + cam.R[6 + j] * dj02 + rot0[j];
      dm1[j] = cam.R[3 + j] * dj11 + cam.R[6 + j] * dj12 + rot1[j];
    }
    float dA = 0.f, dB = 0.f, dC = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float dU = s[i] * (Rg[0][i] * dm0[0] + Rg[1][i] * dm0[1] + Rg[2][i] * dm0[2]);
      const float dV = s[i] * (Rg[0][i] * dm1[0] + Rg[1][i] * dm1[1] + Rg[2][i] * dm1[2]);
      dA += 2.f * U[i] * dU;
      dB += dU * Vv[i] + U[i] * dV;
      dC += 2.f * Vv[i] * dV;
    }
    // d(Sigma'^-1) = -Q dSigma' Q
    const float P00 = qa * dA + qb * dB, P01 = qa * dB + qb * dC, P10 = qb * dA + qc * dB, P11 = qb * dB + qc * dC;
    tg.a[k] = -(P00 * qa + P01 * qb);
    tg.b[k] = -(P00 * qb + P01 * qc);
    tg.c[k] = -(P10 * qb + P11 * qc);
    // colour through the viewing direction: dv = -dc_w
    const float dd = -(dir[0] * dcw[0] + dir[1] * dcw[1] + dir[2] * dcw[2]);
    const float ddir[3] = {(-dcw[0] - dir[0] * dd) * inv, (-dcw[1] - dir[1] * dd) * inv, (-dcw[2] - dir[2] * dd) * inv};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
      tg.col[ch][k] = on[ch] ? Gd[ch].x * ddir[0] + Gd[ch].y * ddir[1] + Gd[ch].z * ddir[2] : 0.f;
  }
}

template <int DEG, bool BF16>
__global__ void __launch_bounds__(128) k_pose_jacobian(gs_map map, const gs_camera* __restrict__ cams, gs_config cfg,
                                                       Ws ws, const int32_t* __restrict__ pix, int32_t n_pix,
                                                       float* __restrict__ J, float* __restrict__ rgb_out) {
  if (ws.counters[kStatus] != 0) return;
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_pix) return;
  const int32_t lin = pix[(int64_t)v * n_pix + k];
  const int64_t out = (int64_t)v * n_pix + k;
  if (lin < 0 || lin >= ws.width * ws.height) {
    for (int i = 0; i < 18; ++i) J[out * 18 + i] = 0.f;
    if (rgb_out) rgb_out[out * 3] = rgb_out[out * 3 + 1] = rgb_out[out * 3 + 2] = 0.f;
    return;
  }
  const int x = lin % ws.width, y = lin / ws.width;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int64_t tile = (int64_t)v * ws.tiles_per_view + (y >> 4) * ws.tiles_x + (x >> 4);
  const uint32_t start = ws.tile_start[tile], cnt = ws.tile_count[tile];
  const Cam cam = load_cam(cams, v);
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  const float lt = __log2f(cfg.alpha_min);
  float T = 1.f, C[3] = {0.f, 0.f, 0.f}, S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, dC[3][6];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) dC[ch][i] = 0.f;
  for (uint32_t j = 0; j < cnt; ++j) {
    const uint32_t gid = ws.sorted_ids[start + j];
    const float4* r = rec + 3 * (int64_t)gid;
    const float4 r0 = r[0], r1 = r[1];
    const Staged sg = stage_gaussian(r0, r1);
    const float p2 = blend_p2(sg.g0, sg.g1, px, py);
    if (!(p2 >= lt)) continue;
    const float araw = ex2_approx(p2);
    const bool clamped = araw > cfg.alpha_max;
    const float al = fminf(cfg.alpha_max, araw);
    const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
    if (Tn < cfg.t_min) break;
    const float4 c = r[2];
    const float col[3] = {c.x, c.y, c.z};
    Tangents tg;
    pose_tangents<DEG, BF16>(map, gid, cam, cfg, ws.width, ws.height, r0, r1, tg);
    const float dx = px - r0.x, dy = py - r0.y;
    const float w = al * T;
    const float inv_om = rcp_approx(__fsub_rn(1.f, al));  // 1 - alpha >= 1 - alpha_max
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float dal = 0.f;
      if (!clamped) {
        const float dpow = (r0.z * dx + r0.w * dy) * tg.mx[i] + (r0.w * dx + r1.x * dy) * tg.my[i] -
                           0.5f * dx * dx * tg.a[i] - dx * dy * tg.b[i] - 0.5f * dy * dy * tg.c[i];
        dal = al * dpow;
      }
      const float dT = -T * S[i];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) dC[ch][i] += tg.col[ch][i] * w + col[ch] * (dal * T + al * dT);
      S[i] += dal * inv_om;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) C[ch] += col[ch] * w;
    T = Tn;
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
    for (int i = 0; i < 6; ++i) J[(out * 3 + ch) * 6 + i] = dC[ch][i] - cfg.bg[ch] * T * S[i];
    if (rgb_out) rgb_out[out * 3 + ch] = C[ch] + T * cfg.bg[ch];
  }
}

template <int DEG, bool BF16>
static cudaError_t launch_jac_t(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                const int32_t* pix, int32_t n_pix, float* J, float* rgb, cudaStream_t st) {
  dim3 grid((unsigned)((n_pix + 127) / 128), (unsigned)ws.views);
  trace_begin(kKPoseJacobian, st);
  k_pose_jacobian<DEG, BF16><<<grid, 128, 0, st>>>(map, cams, cfg, ws, pix, n_pix, J, rgb);
  trace_end(st);
  return cudaGetLastError();
}

cudaError_t launch_pose_jacobian(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                 const int32_t* pix, int32_t n_pix, float* J, float* rgb, cudaStream_t st) {
  const bool bf = map.sh_bf16 != 0;
  switch (map.sh_degree) {
    case 0: return bf ? launch_jac_t<0, true>(map, cams, cfg, ws, pix, n_pix, J, rgb, st) : launch_jac_t<0, false>(map, cams, cfg, ws, pix, n_pix, J, rgb, st);
    case 1: return bf ? launch_jac_t<1, true>(map, cams, cfg, ws, pix, n_pix, J, rgb, st) : launch_jac_t<1, false>(map, cams, cfg, ws, pix, n_pix, J, rgb, st);
    case 2: return bf ? launch_jac_t<2, true>(map, cams, cfg, ws, pix, n_pix, J, rgb, st) : launch_jac_t<2, false>(map, cams, cfg, ws, pix, n_pix, J, rgb, st);
    default: return bf ? launch_jac_t<3, true>(map, cams, cfg, ws, pix, n_pix, J, rgb, st) : launch_jac_t<3, false>(map, cams, cfg, ws, pix, n_pix, J, rgb, st);
  }
}

}  // namespace gsb
