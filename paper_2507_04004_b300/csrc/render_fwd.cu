// Front-to-back compositing of colour, depth and opacity per 16x16 tile
// (arxiv 2507.04004, Eq. alpha, Eq. rendered_rgb, Eq. rendered_depth,
// Eq. rendered_opacity).  One CTA per (view, tile); each thread owns kPPT
// pixels of one column of the tile, so every Gaussian staged in shared memory
// is read once per kPPT pixels.  The tile's depth-sorted Gaussians are staged
// 256 at a time and the CTA stops as soon as every pixel's transmittance is
// exhausted.
#include "gs_internal.h"

namespace gsb {

template <int PPT>
__global__ void __launch_bounds__(256 / PPT) k_render_fwd(gs_config cfg, Ws ws, float* __restrict__ rgb,
                                                          float* __restrict__ depth, float* __restrict__ opac,
                                                          float* __restrict__ t_final,
                                                          uint32_t* __restrict__ n_contrib) {
  constexpr int NT = 256 / PPT;  // threads per tile
  // a thread owns PPT vertically adjacent pixels; a warp covers a 16 x (2 PPT) block
  __shared__ float4 s_g0[256], s_g1[256], s_c[256];
  const int64_t tile = blockIdx.x;
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int tx = t % ws.tiles_x, ty = t / ws.tiles_x;
  const int x = tx * kTile + (threadIdx.x & 15);
  const int yb = ty * kTile + PPT * (threadIdx.x >> 4);
  const float px = (float)x + 0.5f;
  const bool ok_status = ws.counters[kStatus] == 0;
  const uint32_t start = ok_status ? ws.tile_start[tile] : 0u;
  const uint32_t cnt = ok_status ? ws.tile_count[tile] : 0u;
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  const float a_max = cfg.alpha_max, t_min = cfg.t_min;
  const float lt = __log2f(cfg.alpha_min);

  float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT], py[PPT];
  uint32_t last[PPT];
  bool done[PPT];
  bool all_done = true;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f; C0[k] = C1[k] = C2[k] = D[k] = 0.f; last[k] = 0;
    py[k] = (float)(yb + k) + 0.5f;
    done[k] = !(x < ws.width && yb + k < ws.height);
    all_done &= done[k];
  }
  for (uint32_t b0 = 0; b0 < cnt; b0 += 256) {
    if (__syncthreads_count(all_done) == NT) break;
    const uint32_t nb = min(256u, cnt - b0);
    for (uint32_t i = threadIdx.x; i < nb; i += NT) {
      const uint32_t gid = ws.sorted_ids[start + b0 + i];
      const float4* r = rec + 3 * (int64_t)gid;
      const Staged sg = stage_gaussian(r[0], r[1]);
      s_g0[i] = sg.g0;
      s_g1[i] = sg.g1;
      s_c[i] = r[2];
    }
    __syncthreads();
    for (uint32_t j = 0; j < nb && !all_done; ++j) {
      const float4 g0 = s_g0[j], g1 = s_g1[j];
      const ColTerms ct = col_terms(g0, g1, px);
      all_done = true;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const float p2 = col_p2(ct, py[k]);
        if (!done[k]) {
          if (p2 >= lt) {
            const float al = fminf(a_max, exp2f(p2));
            const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, al));
            if (Tn < t_min) {
              done[k] = true;
            } else {
              const float w = __fmul_rn(al, T[k]);
              const float4 c = s_c[j];
              C0[k] = __fmaf_rn(c.x, w, C0[k]);
              C1[k] = __fmaf_rn(c.y, w, C1[k]);
              C2[k] = __fmaf_rn(c.z, w, C2[k]);
              D[k] = __fmaf_rn(g1.z, w, D[k]);
              T[k] = Tn;
              last[k] = b0 + j + 1;
            }
          }
        }
        all_done &= done[k];
      }
    }
    // pixels whose list ended are done only when the whole list is walked
  }
  const int64_t HW = (int64_t)ws.width * ws.height;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int y = yb + k;
    if (!(x < ws.width && y < ws.height)) continue;
    const int64_t p = (int64_t)y * ws.width + x;
    if (rgb) {
      rgb[(3 * (int64_t)v + 0) * HW + p] = __fmaf_rn(T[k], cfg.bg[0], C0[k]);
      rgb[(3 * (int64_t)v + 1) * HW + p] = __fmaf_rn(T[k], cfg.bg[1], C1[k]);
      rgb[(3 * (int64_t)v + 2) * HW + p] = __fmaf_rn(T[k], cfg.bg[2], C2[k]);
    }
    if (depth) depth[v * HW + p] = D[k];
    if (opac) opac[v * HW + p] = 1.f - T[k];
    t_final[v * HW + p] = T[k];
    n_contrib[v * HW + p] = last[k];
  }
}

cudaError_t launch_render_fwd(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                              float* t_final, uint32_t* n_contrib, cudaStream_t st) {
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKRenderFwd, st);
  k_render_fwd<kFwdPPT><<<ntiles, 256 / kFwdPPT, 0, st>>>(cfg, ws, rgb, depth, opac, t_final, n_contrib);
  trace_end(st);
  return cudaGetLastError();
}

}  // namespace gsb
