// Front-to-back compositing of colour, depth and opacity per 16x16 tile
// (arxiv 2507.04004, Eq. alpha, Eq. rendered_rgb, Eq. rendered_depth,
// Eq. rendered_opacity).  One CTA per (view, tile); each thread owns kPPT
// pixels of one column of the tile, so every Gaussian staged in shared memory
// is read once per kPPT pixels.  The tile's depth-sorted Gaussians are staged
// 256 at a time and the CTA stops as soon as every pixel's transmittance is
// exhausted.
//
// The checkpointing variant (CKPT) also records, at the start of every
// 32-Gaussian bucket of the tile's list, each pixel's transmittance and
// accumulated colour and depth, for the per-Gaussian backward of
// Sec. "Per-Gaussian Backpropagation" (bucket b of tile t is record
// (tile_start[t] >> 5) + t + b of the checkpoint array, planes T, C_r, C_g,
// C_b, D of 256 pixels each, pixel index y * 16 + x within the tile).
//
// The counting variant (STATS) composites the same way but writes no image:
// it adds, per view, the number of (pixel, list position) evaluations up to
// each pixel's last contributor, how many of them were blended (the rest
// were skipped below alpha_min), and the list positions the pixels test (up
// to the Gaussian at which each stops, else the whole list) into ckpt
// reinterpreted as uint64 [V][3].
#include "gs_internal.h"

namespace gsb {

template <int PPT, bool CKPT, bool STATS = false>
__global__ void __launch_bounds__(256 / PPT) k_render_fwd(gs_config cfg, Ws ws, float* __restrict__ rgb,
                                                          float* __restrict__ depth, float* __restrict__ opac,
                                                          float* __restrict__ t_final,
                                                          uint32_t* __restrict__ n_contrib,
                                                          float* __restrict__ ckpt) {
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

  // pixels run in vertical pairs (k = 2h, 2h + 1) through packed FP32 pairs
  constexpr int NP = PPT / 2;
  float2 T[NP], C0[NP], C1[NP], C2[NP], D[NP], Y[NP];
  // per-pixel alpha threshold in log2: log2(alpha_min) while the pixel
  // blends, +inf once it is done (or outside the image), so that one
  // comparison decides whether a Gaussian takes part at the pixel
  float thr[PPT];
  uint32_t last[PPT];
  uint32_t n_blend = 0;  // STATS only
  uint32_t stop_at[PPT];  // STATS only: list positions a pixel tests (up to its stop, else the whole list)
  bool all_done = true;
  const float inf = __int_as_float(0x7f800000);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    last[k] = 0;
    const bool out = !(x < ws.width && yb + k < ws.height);
    thr[k] = out ? inf : lt;
    stop_at[k] = out ? 0u : cnt;
    all_done &= out;
  }
#pragma unroll
  for (int h = 0; h < NP; ++h) {
    T[h] = f2(1.f);
    C0[h] = C1[h] = C2[h] = D[h] = f2(0.f);
    Y[h] = make_float2((float)(yb + 2 * h) + 0.5f, (float)(yb + 2 * h + 1) + 0.5f);
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
    // groups of 8 Gaussians; the thread leaves once all its pixels are done,
    // checked after each group (a done pixel takes no part in the ones in between)
    for (uint32_t j0 = 0; j0 < nb && !all_done; j0 += 8) {
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      const uint32_t j = j0 + u;
      if (j >= nb) break;
      if (CKPT && ((b0 + j) & 31u) == 0) {
        float* ck = ckpt + ((int64_t)(start >> 5) + tile + ((b0 + j) >> 5)) * (5 * 256);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const int lp = (threadIdx.x & 15) + 16 * (PPT * (threadIdx.x >> 4) + k);
          const int h = k >> 1;
          const bool hi = k & 1;
          ck[lp] = hi ? T[h].y : T[h].x;
          ck[256 + lp] = hi ? C0[h].y : C0[h].x;
          ck[512 + lp] = hi ? C1[h].y : C1[h].x;
          ck[768 + lp] = hi ? C2[h].y : C2[h].x;
          ck[1024 + lp] = hi ? D[h].y : D[h].x;
        }
      }
      const float4 g0 = s_g0[j], g1 = s_g1[j];
      const ColTerms ct = col_terms(g0, g1, px);
      const float4 c = s_c[j];
      const float2 cr = f2(c.x), cg = f2(c.y), cb = f2(c.z), dep = f2(g1.z);
      const uint32_t nxt = b0 + j + 1;
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        // a pixel blends this Gaussian unless it is done, below alpha_min, or
        // would drop under t_min (then it is done and this Gaussian is not blended)
        const float2 p2 = col_p2x2(ct, Y[h]);
        const bool a0 = p2.x >= thr[2 * h], a1 = p2.y >= thr[2 * h + 1];
        const float2 al = make_float2(fminf(a_max, ex2_approx(p2.x)), fminf(a_max, ex2_approx(p2.y)));
        const float2 Tc = mul2(T[h], fma2(al, f2(-1.f), f2(1.f)));
        const bool s0 = a0 & (Tc.x < t_min), s1 = a1 & (Tc.y < t_min);
        const bool k0 = a0 & !s0, k1 = a1 & !s1;
        thr[2 * h] = s0 ? inf : thr[2 * h];
        thr[2 * h + 1] = s1 ? inf : thr[2 * h + 1];
        // alpha of a blended pixel, 0 otherwise: T (1 - 0) = T leaves the others as they are
        const float2 ak = make_float2(k0 ? al.x : 0.f, k1 ? al.y : 0.f);
        const float2 w = mul2(ak, T[h]);
        C0[h] = fma2(cr, w, C0[h]);
        C1[h] = fma2(cg, w, C1[h]);
        C2[h] = fma2(cb, w, C2[h]);
        D[h] = fma2(dep, w, D[h]);
        T[h] = mul2(T[h], fma2(ak, f2(-1.f), f2(1.f)));
        last[2 * h] = k0 ? nxt : last[2 * h];
        last[2 * h + 1] = k1 ? nxt : last[2 * h + 1];
        if (STATS) {
          n_blend += (uint32_t)k0 + (uint32_t)k1;
          stop_at[2 * h] = s0 ? nxt : stop_at[2 * h];
          stop_at[2 * h + 1] = s1 ? nxt : stop_at[2 * h + 1];
        }
      }
    }
      all_done = true;
#pragma unroll
      for (int k = 0; k < PPT; ++k) all_done &= thr[k] == inf;
    }
    // pixels whose list ended are done only when the whole list is walked
  }
  const int64_t HW = (int64_t)ws.width * ws.height;
  if (STATS) {
    unsigned long long ev = 0, bl = n_blend, need = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      ev += last[k];
      need += stop_at[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(kFull, ev, o);
      bl += __shfl_xor_sync(kFull, bl, o);
      need += __shfl_xor_sync(kFull, need, o);
    }
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ckpt) + 3 * v;
    if ((threadIdx.x & 31) == 0 && need) {
      atomicAdd(counts, ev);
      atomicAdd(counts + 1, bl);
      atomicAdd(counts + 2, need);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int y = yb + k;
    if (!(x < ws.width && y < ws.height)) continue;
    const int64_t p = (int64_t)y * ws.width + x;
    const int h = k >> 1;
    const bool hi = k & 1;
    const float Tk = hi ? T[h].y : T[h].x;
    if (rgb) {
      rgb[(3 * (int64_t)v + 0) * HW + p] = __fmaf_rn(Tk, cfg.bg[0], hi ? C0[h].y : C0[h].x);
      rgb[(3 * (int64_t)v + 1) * HW + p] = __fmaf_rn(Tk, cfg.bg[1], hi ? C1[h].y : C1[h].x);
      rgb[(3 * (int64_t)v + 2) * HW + p] = __fmaf_rn(Tk, cfg.bg[2], hi ? C2[h].y : C2[h].x);
    }
    if (depth) depth[v * HW + p] = hi ? D[h].y : D[h].x;
    if (opac) opac[v * HW + p] = 1.f - Tk;
    t_final[v * HW + p] = Tk;
    n_contrib[v * HW + p] = last[k];
  }
}

cudaError_t launch_render_fwd(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                              float* t_final, uint32_t* n_contrib, cudaStream_t st) {
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKRenderFwd, st);
  k_render_fwd<kFwdPPT, false><<<ntiles, 256 / kFwdPPT, 0, st>>>(cfg, ws, rgb, depth, opac, t_final, n_contrib,
                                                                  nullptr);
  trace_end(st);
  return cudaGetLastError();
}

cudaError_t launch_render_fwd_ckpt(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                                   float* t_final, uint32_t* n_contrib, float* ckpt, cudaStream_t st) {
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKRenderFwdCkpt, st);
  k_render_fwd<kFwdPPT, true><<<ntiles, 256 / kFwdPPT, 0, st>>>(cfg, ws, rgb, depth, opac, t_final, n_contrib, ckpt);
  trace_end(st);
  return cudaGetLastError();
}

}  // namespace gsb

namespace gsb {

cudaError_t launch_blend_counts(const gs_config& cfg, const Ws& ws, unsigned long long* counts, cudaStream_t st) {
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)ws.views * 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_render_fwd<kFwdPPT, false, true><<<ntiles, 256 / kFwdPPT, 0, st>>>(cfg, ws, nullptr, nullptr, nullptr, nullptr,
                                                                        nullptr, reinterpret_cast<float*>(counts));
  return cudaGetLastError();
}

}  // namespace gsb
