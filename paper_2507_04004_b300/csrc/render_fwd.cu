// Front-to-back compositing of colour, depth and opacity per 16x16 tile
// (arxiv 2507.04004, Eq. alpha, Eq. rendered_rgb, Eq. rendered_depth,
// Eq. rendered_opacity).  One CTA per (view, tile), one thread per pixel; the
// tile's depth-sorted Gaussians are staged into shared memory 256 at a time
// and the CTA stops as soon as every pixel's transmittance is exhausted.
#include "gs_internal.h"

namespace gsb {

__global__ void __launch_bounds__(256) k_render_fwd(gs_config cfg, Ws ws, float* __restrict__ rgb,
                                                    float* __restrict__ depth, float* __restrict__ opac,
                                                    float* __restrict__ t_final, uint32_t* __restrict__ n_contrib) {
  __shared__ float4 s_r0[256], s_r1[256], s_r2[256];
  const int64_t tile = blockIdx.x;
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int tx = t % ws.tiles_x, ty = t / ws.tiles_x;
  const int x = tx * kTile + (threadIdx.x & 15), y = ty * kTile + (threadIdx.x >> 4);
  const bool inside = x < ws.width && y < ws.height;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const bool ok_status = ws.counters[kStatus] == 0;
  const uint32_t start = ok_status ? ws.tile_start[tile] : 0u;
  const uint32_t cnt = ok_status ? ws.tile_count[tile] : 0u;
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  const float a_min = cfg.alpha_min, a_max = cfg.alpha_max, t_min = cfg.t_min;

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  uint32_t last = 0;
  bool done = !inside;
  for (uint32_t b0 = 0; b0 < cnt; b0 += 256) {
    if (__syncthreads_count(done) == 256) break;
    const uint32_t nb = min(256u, cnt - b0);
    if (threadIdx.x < nb) {
      const uint32_t gid = ws.sorted_ids[start + b0 + threadIdx.x];
      const float4* r = rec + 3 * (int64_t)gid;
      s_r0[threadIdx.x] = r[0];
      s_r1[threadIdx.x] = r[1];
      s_r2[threadIdx.x] = r[2];
    }
    __syncthreads();
    if (!done) {
      for (uint32_t j = 0; j < nb; ++j) {
        const AlphaEval ev = eval_alpha(s_r0[j], s_r1[j], px, py, a_min, a_max);
        if (!ev.pass) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, ev.alpha));
        if (Tn < t_min) { done = true; break; }
        const float w = __fmul_rn(ev.alpha, T);
        const float4 c = s_r2[j];
        C0 = __fmaf_rn(c.x, w, C0);
        C1 = __fmaf_rn(c.y, w, C1);
        C2 = __fmaf_rn(c.z, w, C2);
        D = __fmaf_rn(s_r1[j].z, w, D);
        T = Tn;
        last = b0 + j + 1;
      }
    }
  }
  if (!inside) return;
  const int64_t HW = (int64_t)ws.width * ws.height;
  const int64_t p = (int64_t)y * ws.width + x;
  if (rgb) {
    rgb[(3 * (int64_t)v + 0) * HW + p] = __fmaf_rn(T, cfg.bg[0], C0);
    rgb[(3 * (int64_t)v + 1) * HW + p] = __fmaf_rn(T, cfg.bg[1], C1);
    rgb[(3 * (int64_t)v + 2) * HW + p] = __fmaf_rn(T, cfg.bg[2], C2);
  }
  if (depth) depth[v * HW + p] = D;
  if (opac) opac[v * HW + p] = 1.f - T;
  t_final[v * HW + p] = T;
  n_contrib[v * HW + p] = last;
}

cudaError_t launch_render_fwd(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                              float* t_final, uint32_t* n_contrib, cudaStream_t st) {
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKRenderFwd, st);
  k_render_fwd<<<ntiles, 256, 0, st>>>(cfg, ws, rgb, depth, opac, t_final, n_contrib);
  trace_end(st);
  return cudaGetLastError();
}

}  // namespace gsb
