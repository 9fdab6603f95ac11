// Backward pass of the rasterizer (arxiv 2507.04004):
//   - pixel adjoints of the depth-regularised loss of Eq. depth_loss
//     (L1 colour mean plus the opacity-normalised L1 depth term on the valid
//     LiDAR pixels), fused into the blend backward;
//   - the adjoint of front-to-back compositing (Eq. rendered_rgb,
//     rendered_depth, rendered_opacity) per tile, walking each pixel's
//     contributors back to front and recovering the transmittance before each
//     Gaussian from the final one, T_i = T_{i+1} / (1 - alpha_i), so no
//     per-pixel lists are stored;
//   - per-Gaussian 2D adjoints reduced across each warp with shuffles, then
//     across the CTA in shared memory, then one vector atomic per
//     (Gaussian, tile) into the workspace;
//   - the chain through the projection (Sec. "3D Gaussian Splatting
//     Representation") to mean, log-scale, quaternion, opacity logit and SH,
//     and the per-view pose derivative under T Exp(xi) (Eq. 3dgs_jacobi).
#include <type_traits>

#include "gs_internal.h"
#include "radix.cuh"

namespace gsb {

// Count of valid LiDAR pixels (D_s > 0) per view: |M_d| of Eq. depth_loss.
__global__ void __launch_bounds__(256) k_count_depth(const float* __restrict__ tgt_depth, int64_t hw,
                                                     float* view_stats) {
  const int v = blockIdx.y;
  uint32_t c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x)
    c += tgt_depth[v * hw + i] > 0.f ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  __shared__ uint32_t s[8];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int i = 0; i < 8; ++i) tot += s[i];
    if (tot) atomicAdd(view_stats + 4 * v + 1, (float)tot);
  }
}

// The backward's per-Gaussian sums leave the warp through shared memory:
// every lane writes its 10 partial sums of a Gaussian to s_part[slot][lane]
// (rows of 12 floats, so a quarter-warp's 16-byte stores hit 32 distinct
// banks), and every kRedGroup Gaussians the warp reduces the group at once,
// 8 lanes per Gaussian (lane = 8 g + s, each lane summing the rows of lanes
// s, s + 8, s + 16, s + 24), then a reduce-scatter over the 8 lanes.
constexpr int kRedGroup = 4;
constexpr int kRedRow = 12;

// Reduce-scatter of 10 values over the 8 lanes s = lane & 7 of a group
// (butterflies over lane bits 2, 1, 0).  Afterwards lane s holds in y0 / y1
// the 8-lane sums of values: s=0: 0, 1; s=1: 2; s=2: 3, 4; s=4: 5, 6;
// s=5: 7; s=6: 8, 9 (the other slots hold nothing meaningful).
__device__ __forceinline__ void group8_reduce_scatter10(const float v[10], int s, float* y0, float* y1) {
  const bool b2 = s & 4, b1 = s & 2, b0 = s & 1;
  float w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float keep = b2 ? v[i + 5] : v[i];
    const float send = b2 ? v[i] : v[i + 5];
    w[i] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  float x[3];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b1 ? w[i + 3] : w[i];
    const float send = b1 ? w[i] : w[i + 3];
    x[i] = keep + __shfl_xor_sync(kFull, send, 2);
  }
  x[2] = (b1 ? 0.f : w[2]) + __shfl_xor_sync(kFull, b1 ? w[2] : 0.f, 2);
  *y0 = (b0 ? x[2] : x[0]) + __shfl_xor_sync(kFull, b0 ? x[0] : x[2], 1);
  *y1 = (b0 ? 0.f : x[1]) + __shfl_xor_sync(kFull, b0 ? x[1] : 0.f, 1);
}

// A colour byte c as the target value c / 255, correctly rounded: the
// reciprocal product q = c r (r = 1/255 rounded) with one residual
// correction q + (c - 255 q) r by fused multiply-adds (Markstein's method).
// For the 256 byte values this equals the IEEE quotient exactly (checked
// against the host's division for every c), with no division in the kernel.
__device__ __forceinline__ float byte_unit(uint8_t b) {
  const float c = (float)b, r = 1.f / 255.f;
  const float q = __fmul_rn(c, r);
  return __fmaf_rn(__fmaf_rn(-q, 255.f, c), r, q);
}

// One (view, tile) item of the blend backward.  DEP: the pixel adjoints of
// depth and opacity may be nonzero (a depth loss or the caller's depth /
// opacity adjoints); without them (colour-only losses, e.g. tracking) they
// and their terms are left out at compile time.
template <bool FUSED, bool DEP, int PPT, bool U8>
__device__ __forceinline__ void bwd_tile(const gs_config& cfg, const Ws& ws, const BwdArgs& a, const int64_t tile) {
  constexpr int NT = 256 / PPT;  // threads per tile
  constexpr int NW = NT / 32;    // warps per tile
  // a thread owns PPT vertically adjacent pixels; a warp covers a 16 x (2 PPT) block
  // Gaussians staged per batch (fewer without the depth terms, whose
  // lighter register use lets more CTAs share an SM's shared memory)
  constexpr int NB = DEP ? kBwdBatch : kBwdBatch * 3 / 4;
  __shared__ float4 s_g0[NB], s_g1[NB], s_c[NB];
  __shared__ uint32_t s_gid[NB];
  static_assert(NW == 1, "the per-Gaussian sums are reduced by the tile's only warp");
  __shared__ __align__(16) float s_part[kRedGroup][32][kRedRow];
  __shared__ float s_red[NW];
  __shared__ uint32_t s_max[NW];
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int tx = t % ws.tiles_x, ty = t / ws.tiles_x;
  const int x = tx * kTile + (threadIdx.x & 15);
  const int yb = ty * kTile + PPT * (threadIdx.x >> 4);
  const float px = (float)x + 0.5f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t HW = (int64_t)ws.width * ws.height;
  const uint32_t start = ws.tile_start[tile];
  const uint32_t cnt = ws.tile_count[tile];
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  float4* adj = ws.adjoints + 3 * (int64_t)v * ws.n;

  // ---- per-pixel adjoints (dL/dC, dL/dD, dL/dO) and loss
  float gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gO[PPT], T[PPT], py[PPT];
  // S = adjoint-weighted value of everything behind the current Gaussian:
  // sum over later contributors j of (gC.c_j + gD d_j + gO) alpha_j T_j / T_next, plus gC.bg.
  // The walk keeps S - gO instead: it obeys the same recursion
  // S_i = alpha_i x_i + (1 - alpha_i) S_{i+1} with gO dropped from every
  // value x_i, so gO needs no register of its own.
  float S[PPT];
  uint32_t last[PPT];
  float loss = 0.f;
  uint32_t mx = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int y = yb + k;
    py[k] = (float)y + 0.5f;
    gC0[k] = gC1[k] = gC2[k] = gD[k] = gO[k] = 0.f;
    T[k] = 1.f;
    last[k] = 0;
    S[k] = 0.f;
    if (!(x < ws.width && y < ws.height)) continue;
    const int64_t p = (int64_t)y * ws.width + x;
    T[k] = a.t_final[v * HW + p];
    last[k] = min(a.n_contrib[v * HW + p], cnt);  // never walk past the tile's list
    if (FUSED) {
      // the colour target: FP32 planes, or (U8) the 8-bit images as c / 255
      auto tgt = [&](int64_t i) { return U8 ? byte_unit(a.tgt_rgb8[i]) : a.tgt_rgb[i]; };
      const float inv3hw = a.w_rgb / (3.f * (float)HW);
      float r = a.rgb[(3 * (int64_t)v + 0) * HW + p] - tgt((3 * (int64_t)v + 0) * HW + p);
      gC0[k] = inv3hw * (float)((r > 0.f) - (r < 0.f)); loss += inv3hw * fabsf(r);
      r = a.rgb[(3 * (int64_t)v + 1) * HW + p] - tgt((3 * (int64_t)v + 1) * HW + p);
      gC1[k] = inv3hw * (float)((r > 0.f) - (r < 0.f)); loss += inv3hw * fabsf(r);
      r = a.rgb[(3 * (int64_t)v + 2) * HW + p] - tgt((3 * (int64_t)v + 2) * HW + p);
      gC2[k] = inv3hw * (float)((r > 0.f) - (r < 0.f)); loss += inv3hw * fabsf(r);
      if (DEP && a.tgt_depth && a.w_depth != 0.f) {
        const float ds = a.tgt_depth[v * HW + p];
        const float O = a.opac[v * HW + p], Dp = a.depth[v * HW + p];
        const float nd = ws.view_stats[4 * v + 1];
        if (ds > 0.f && O > 0.f && nd > 0.f) {
          const float rd = Dp / O - ds;
          const float sg = (float)((rd > 0.f) - (rd < 0.f));
          gD[k] = a.w_depth * sg / (O * nd);
          gO[k] = -a.w_depth * sg * Dp / (O * O * nd);
          loss += a.w_depth * fabsf(rd) / nd;
        }
      }
      // further pixel adjoints of other loss terms (e.g. D-SSIM) add to the fused ones
      if (a.dl_drgb) {
        gC0[k] += a.dl_drgb[(3 * (int64_t)v + 0) * HW + p];
        gC1[k] += a.dl_drgb[(3 * (int64_t)v + 1) * HW + p];
        gC2[k] += a.dl_drgb[(3 * (int64_t)v + 2) * HW + p];
      }
      if (DEP && a.dl_ddepth) gD[k] += a.dl_ddepth[v * HW + p];
      if (DEP && a.dl_dopac) gO[k] += a.dl_dopac[v * HW + p];
    } else {
      if (a.dl_drgb) {
        gC0[k] = a.dl_drgb[(3 * (int64_t)v + 0) * HW + p];
        gC1[k] = a.dl_drgb[(3 * (int64_t)v + 1) * HW + p];
        gC2[k] = a.dl_drgb[(3 * (int64_t)v + 2) * HW + p];
      }
      if (DEP && a.dl_ddepth) gD[k] = a.dl_ddepth[v * HW + p];
      if (DEP && a.dl_dopac) gO[k] = a.dl_dopac[v * HW + p];
    }
    mx = max(mx, last[k]);
    S[k] = gC0[k] * cfg.bg[0] + gC1[k] * cfg.bg[1] + gC2[k] * cfg.bg[2] - gO[k];
  }
  // CTA reductions: loss sum and the longest contributor prefix
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    loss += __shfl_xor_sync(kFull, loss, o);
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if (lane == 0) { s_red[warp] = loss; s_max[warp] = mx; }
  __syncthreads();
  uint32_t max_last = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) max_last = max(max_last, s_max[i]);
  if (FUSED && a.loss && threadIdx.x == 0) {
    float tot = 0.f;
    for (int i = 0; i < NW; ++i) tot += s_red[i];
    if (tot != 0.f) atomicAdd(a.loss + v, tot);
  }

  // ---- back-to-front walk over vertical pixel pairs (k = 2h, 2h + 1)
  constexpr int NP = PPT / 2;
  float2 C0[NP], C1[NP], C2[NP], GD[NP], T2[NP], S2[NP], Y[NP];
#pragma unroll
  for (int h = 0; h < NP; ++h) {
    C0[h] = make_float2(gC0[2 * h], gC0[2 * h + 1]);
    C1[h] = make_float2(gC1[2 * h], gC1[2 * h + 1]);
    C2[h] = make_float2(gC2[2 * h], gC2[2 * h + 1]);
    GD[h] = make_float2(gD[2 * h], gD[2 * h + 1]);
    T2[h] = make_float2(T[2 * h], T[2 * h + 1]);
    Y[h] = make_float2(py[2 * h], py[2 * h + 1]);
    S2[h] = make_float2(S[2 * h], S[2 * h + 1]);
  }
  const float a_max = cfg.alpha_max;
  const float lt = __log2f(cfg.alpha_min);
  const float clamp_from = __log2f(cfg.alpha_max) - 1e-4f;
  for (int64_t end = max_last; end > 0; end -= NB) {
    const int64_t beg = end > NB ? end - NB : 0;
    const int nb = (int)(end - beg);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += NT) {
      const uint32_t gid = ws.sorted_ids[start + beg + i];
      s_gid[i] = gid;
      const float4* r = rec + 3 * (int64_t)gid;
      const Staged sg = stage_gaussian(r[0], r[1]);
      s_g0[i] = sg.g0;
      s_g1[i] = sg.g1;
      s_c[i] = r[2];
    }
    __syncthreads();
    // groups of kRedGroup Gaussians, back to front; slot gs of a group holds
    // staged Gaussian j0 - gs
    for (int j0 = nb - 1; j0 >= 0; j0 -= kRedGroup) {
#pragma unroll
    for (int gs = 0; gs < kRedGroup; ++gs) {
      const int j = j0 - gs;
      if (j < 0) break;
      const float4 g0 = s_g0[j], g1 = s_g1[j];
      const uint32_t pos = (uint32_t)(beg + j);
      const float dx = px - g0.x;
      const ColTerms ct = col_terms(g0, g1, px);
      float2 ea[NP];  // o 2^p2 where the pixel takes part, 0 elsewhere
      bool any = false;
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        const float2 p2 = col_p2x2(ct, Y[h]);
        const bool a0 = (pos < last[2 * h]) & (p2.x >= lt);
        const bool a1 = (pos < last[2 * h + 1]) & (p2.y >= lt);
        const float e0 = ex2_approx(p2.x), e1 = ex2_approx(p2.y);
        ea[h] = make_float2(a0 ? e0 : 0.f, a1 ? e1 : 0.f);
        any |= a0 | a1;
      }
      float val[10];  // this lane's partial sums of the Gaussian (zero when no pixel of the warp takes part)
      if (__any_sync(kFull, any)) {
      // Per-Gaussian sums over this thread's pixels.  With dp = dL/dpower
      // (power = -q/2, zero where alpha is clamped), the conic and opacity
      // gradients need only the moments of dp; their constant factors are
      // applied once per Gaussian when the CTA's sums are flushed:
      //   val[0..5] = sum dp dx, dp dy, dp dx^2, dp dx dy, dp dy^2, dp
      //   val[6..9] = sum gD w, gC w (w = alpha T)
      // The thread's pixels share one column (dx) and sit at dy = dy0 + k, so
      // the six moments follow from m_i = sum k^i dp, i = 0, 1, 2.
      // Pixels run in vertical pairs, branch-free: an inactive pixel gets
      // alpha = 0, for which every update below leaves its state unchanged.
      const float4 c = s_c[j];
      const float2 cr = f2(c.x), cg = f2(c.y), cb = f2(c.z), dep = f2(g1.z);
      float2 v6 = f2(0.f), v7 = f2(0.f), v8 = f2(0.f), v9 = f2(0.f);
      float2 M0 = f2(0.f), M1 = f2(0.f), M2 = f2(0.f);
      auto walk = [&](auto clamp) {
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        float2 al, ag;
        if (decltype(clamp)::value) {
          al = make_float2(fminf(a_max, ea[h].x), fminf(a_max, ea[h].y));
          // alpha = o exp(power): dL/dpower = dL/dalpha alpha, zero where alpha is clamped
          ag = make_float2(ea[h].x > a_max ? 0.f : al.x, ea[h].y > a_max ? 0.f : al.y);
        } else {
          al = ea[h];
          ag = al;
        }
        // 1 - alpha >= 0.01; exactly 1 where alpha = 0, whose reciprocal leaves T as it is
        // (up to the approximate reciprocal's one-ulp bound)
        const float2 om = fma2(al, f2(-1.f), f2(1.f));
        // transmittance in front of this Gaussian
        T2[h] = mul2(T2[h], make_float2(rcp_approx(om.x), rcp_approx(om.y)));
        const float2 w = mul2(al, T2[h]);
        const float2 gx = DEP ? fma2(C0[h], cr, fma2(C1[h], cg, fma2(C2[h], cb, mul2(GD[h], dep))))
                              : fma2(C0[h], cr, fma2(C1[h], cg, mul2(C2[h], cb)));
        const float2 e = fma2(S2[h], f2(-1.f), gx);
        S2[h] = fma2(al, e, S2[h]);
        if (DEP) v6 = fma2(GD[h], w, v6);
        v7 = fma2(C0[h], w, v7);
        v8 = fma2(C1[h], w, v8);
        v9 = fma2(C2[h], w, v9);
        // dp = dL/dalpha alpha with dL/dalpha = T e; unclamped, that is w e
        const float2 dp = decltype(clamp)::value ? mul2(mul2(T2[h], e), ag) : mul2(w, e);
        M0 = add2(M0, dp);
        M1 = fma2(dp, make_float2((float)(2 * h), (float)(2 * h + 1)), M1);
        M2 = fma2(dp, make_float2((float)(4 * h * h), (float)((2 * h + 1) * (2 * h + 1))), M2);
      }
      };
      // the clamp of alpha can act only where the opacity nearly reaches
      // alpha_max (per Gaussian, warp-uniform, with a margin for the rounding
      // of p2): other Gaussians take the path without it
      if (g1.y > clamp_from) walk(std::true_type{});
      else walk(std::false_type{});
      const float m0 = M0.x + M0.y, m1 = M1.x + M1.y, m2 = M2.x + M2.y;
      const float dy0 = Y[0].x - g0.y;
      const float sy = fmaf(dy0, m0, m1);  // sum dp dy
      val[0] = dx * m0;
      val[1] = sy;
      val[2] = dx * val[0];
      val[3] = dx * sy;
      val[4] = fmaf(dy0, sy + m1, m2);     // dy0^2 m0 + 2 dy0 m1 + m2
      val[5] = m0;
      val[6] = v6.x + v6.y;
      val[7] = v7.x + v7.y;
      val[8] = v8.x + v8.y;
      val[9] = v9.x + v9.y;
      } else {
#pragma unroll
        for (int q = 0; q < 10; ++q) val[q] = 0.f;
      }
      float* row = &s_part[gs][lane][0];
      *reinterpret_cast<float4*>(row) = make_float4(val[0], val[1], val[2], val[3]);
      *reinterpret_cast<float4*>(row + 4) = make_float4(val[4], val[5], val[6], val[7]);
      *reinterpret_cast<float2*>(row + 8) = make_float2(val[8], val[9]);
    }
      {
        const int filled = min(kRedGroup, j0 + 1);  // Gaussians of this group
        __syncwarp();
        const int g = lane >> 3, s = lane & 7;
        const bool mine = g < filled;
        float2 acc2[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) acc2[q] = f2(0.f);
        if (mine) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float* src = &s_part[g][s + 8 * k][0];
            const float4 u0 = *reinterpret_cast<const float4*>(src);
            const float4 u1 = *reinterpret_cast<const float4*>(src + 4);
            const float2 u2 = *reinterpret_cast<const float2*>(src + 8);
            acc2[0] = add2(acc2[0], make_float2(u0.x, u0.y));
            acc2[1] = add2(acc2[1], make_float2(u0.z, u0.w));
            acc2[2] = add2(acc2[2], make_float2(u1.x, u1.y));
            acc2[3] = add2(acc2[3], make_float2(u1.z, u1.w));
            acc2[4] = add2(acc2[4], u2);
          }
        }
        const float acc[10] = {acc2[0].x, acc2[0].y, acc2[1].x, acc2[1].y, acc2[2].x,
                               acc2[2].y, acc2[3].x, acc2[3].y, acc2[4].x, acc2[4].y};
        float y0, y1;
        group8_reduce_scatter10(acc, s, &y0, &y1);
        // gather each atomic's values into one lane: s=0 takes values 2 (from
        // s=1) and 3 (s=2); s=4 takes value 4 (s=2); s=6 takes value 7 (s=5)
        const float h1 = __shfl_sync(kFull, y0, lane + (s == 0 ? 1 : (s == 6 ? -1 : 0)));
        const float h2 = __shfl_sync(kFull, y0, lane + (s == 0 ? 2 : 0));
        const float h3 = __shfl_sync(kFull, y1, lane - (s == 4 ? 2 : 0));
        // lanes s = 0, 4, 6 add parts 0, 1, 2 of the Gaussian's adjoint record
        // (branch-free: the three roles differ only in selects)
        const int jg = mine ? j0 - g : j0;
        const float4 q0 = s_g0[jg], q1 = s_g1[jg];
        const uint32_t gid = s_gid[jg];
        const bool r0 = s == 0, r1 = s == 4;
        // d power / d mx = a dx + b dy, with a = -2 ln2 ha, b = -ln2 hb, c = -2 ln2 hc;
        // d power / d(a, b, c) = (-dx^2/2, -dx dy, -dy^2/2); d alpha / d o = alpha / o
        const float gmx = -kLn2 * (2.f * q0.z * y0 + q0.w * y1);
        const float gmy = -kLn2 * (q0.w * y0 + 2.f * q1.x * y1);
        const float4 out = make_float4(r0 ? gmx : (r1 ? -0.5f * h3 : h1), r0 ? gmy : (r1 ? y0 * q1.w : y0),
                                       r0 ? -0.5f * h1 : y1, r0 ? -h2 : 0.f);
        if (mine && (r0 || r1 || s == 6) && (out.x != 0.f || out.y != 0.f || out.z != 0.f || out.w != 0.f))
          red_add4(adj + 3 * (int64_t)gid + (s + 2) / 4, out);
        __syncwarp();
      }
    }
  }
}

// Work list of the blend backward.  A tile's work is its longest contributor
// prefix w (the maximum of its pixels' n_contrib: the list positions its
// backward walks); k_tile_work puts every (view, tile) item into one of
// kWorkClasses classes, class floor(6 log2(w + 1)) (classes grow by 2^(1/6)),
// and CTA b of the backward takes item b of the classes' items, longest
// class first, so the last CTAs to start are short and the launch ends
// evenly.  Order inside a class is arbitrary; any order gives the same
// gradients up to the summation order of float atomics.
__device__ __forceinline__ uint32_t work_class(uint32_t w) {
  return (uint32_t)min(kWorkClasses - 1, (int)(6.f * __log2f((float)w + 1.f)));
}

constexpr int kWorkThreads = 1024;                  // threads of one CTA of k_tile_work
constexpr int kWorkPerWarp = 4;                     // items per warp, their loads in flight together
constexpr int kWorkItemsPerCta = kWorkThreads / 32 * kWorkPerWarp;

// Per CTA kWorkItemsPerCta (view, tile) items, kWorkPerWarp per warp: each
// item's work from the tile's n_contrib words (a half-warp reads one pixel
// row, 16 consecutive words); the CTA's items counted per class in shared
// memory, one reservation per class of the CTA, then every item written to
// its class list (fill counts cleared before).  With tgt_depth given, the
// same pass counts the valid LiDAR pixels (D_s > 0) of every view: |M_d| of
// Eq. depth_loss, added to view_stats (cleared before).
__global__ void __launch_bounds__(kWorkThreads) k_tile_work(Ws ws, const uint32_t* __restrict__ n_contrib,
                                                            const float* __restrict__ tgt_depth) {
  __shared__ uint32_t s_cnt[kWorkClasses], s_base[kWorkClasses];
  __shared__ uint32_t s_cls[kWorkItemsPerCta], s_rank[kWorkItemsPerCta];
  __shared__ uint32_t s_depth[2];  // valid depth pixels of the CTA's first view and the next one
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t items = (int64_t)ws.views * ws.tiles_per_view;
  const int64_t first = (int64_t)blockIdx.x * kWorkItemsPerCta + (int64_t)warp * kWorkPerWarp;
  const int v_cta = (int)((int64_t)blockIdx.x * kWorkItemsPerCta / ws.tiles_per_view);
  for (int c = threadIdx.x; c < kWorkClasses; c += kWorkThreads) s_cnt[c] = 0;
  if (threadIdx.x < 2) s_depth[threadIdx.x] = 0;
  uint32_t w[kWorkPerWarp], nd[kWorkPerWarp];
#pragma unroll
  for (int q = 0; q < kWorkPerWarp; ++q) {
    w[q] = 0;
    nd[q] = 0;
    const int64_t item = first + q;
    if (item >= items) continue;
    const int v = (int)(item / ws.tiles_per_view);
    const int t = (int)(item - (int64_t)v * ws.tiles_per_view);
    const int tx = t % ws.tiles_x, ty = t / ws.tiles_x;
    const int x = tx * kTile + (lane & 15);
#pragma unroll
    for (int r = 0; r < kTile; r += 2) {
      const int y = ty * kTile + r + (lane >> 4);
      if (x < ws.width && y < ws.height) {
        const int64_t p = ((int64_t)v * ws.height + y) * ws.width + x;
        w[q] = max(w[q], n_contrib[p]);
        if (tgt_depth) nd[q] += tgt_depth[p] > 0.f ? 1u : 0u;
      }
    }
  }
  __syncthreads();  // s_cnt, s_depth cleared
#pragma unroll
  for (int q = 0; q < kWorkPerWarp; ++q) {
    const uint32_t m = __reduce_max_sync(kFull, w[q]);
    const uint32_t d = tgt_depth ? __reduce_add_sync(kFull, nd[q]) : 0u;
    const int64_t item = first + q;
    if (lane == 0 && item < items) {
      const int li = warp * kWorkPerWarp + q;
      const uint32_t c = work_class(min(m, ws.tile_count[item]));
      s_cls[li] = c;
      s_rank[li] = atomicAdd(&s_cnt[c], 1u);
      if (d) {
        const int v = (int)(item / ws.tiles_per_view);
        if (v - v_cta < 2) atomicAdd(&s_depth[v - v_cta], d);
        else atomicAdd(ws.view_stats + 4 * v + 1, (float)d);  // views of fewer tiles than a CTA's items
      }
    }
  }
  __syncthreads();
  if (tgt_depth && threadIdx.x < 2 && s_depth[threadIdx.x] && v_cta + (int)threadIdx.x < ws.views)
    atomicAdd(ws.view_stats + 4 * (v_cta + threadIdx.x) + 1, (float)s_depth[threadIdx.x]);
  for (int c = threadIdx.x; c < kWorkClasses; c += kWorkThreads)
    if (s_cnt[c]) s_base[c] = atomicAdd(ws.work_fill + c, s_cnt[c]);
  __syncthreads();
  for (int li = threadIdx.x; li < kWorkItemsPerCta; li += kWorkThreads) {
    const int64_t it = (int64_t)blockIdx.x * kWorkItemsPerCta + li;
    if (it < items) {
      const uint32_t c = s_cls[li];
      ws.work_lists[(int64_t)c * items + s_base[c] + s_rank[li]] = (uint32_t)it;
    }
  }
}

// The blend backward over the work list: CTA b takes item b of the
// sequence of the classes' items, longest class first (the hardware starts
// CTAs in index order); when the lists do not hold every item once (not
// filled since the last binning), item b is tile b.
template <bool FUSED, bool DEP, int PPT, bool U8>
__global__ void __launch_bounds__(256 / PPT, PPT == 8 ? (DEP ? 16 : 18) : 2048 / (256 / PPT) / 2)
    k_render_bwd(gs_config cfg, Ws ws, BwdArgs a) {
  __shared__ uint32_t s_item;
  if (ws.counters[kStatus] != 0) return;
  const int64_t items = (int64_t)ws.views * ws.tiles_per_view;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    uint32_t k = blockIdx.x, item = k;
    uint32_t run = 0, total = 0;
    bool found = false;
#pragma unroll
    for (int h = 0; h < kWorkClasses; h += 32) {  // classes longest first, 32 at a time
      const int c = kWorkClasses - 1 - (h + lane);
      const uint32_t f = ws.work_fill[c];
      const uint32_t incl = warp_incl_scan(f, lane) + run;
      // the first lane whose running count passes k holds k's class
      const unsigned m = __ballot_sync(kFull, k < incl);
      if (!found && m) {
        const int l = __ffs(m) - 1;
        const uint32_t before = __shfl_sync(kFull, incl - f, l);
        const int cc = kWorkClasses - 1 - (h + l);
        item = ws.work_lists[(int64_t)cc * items + (k - before)];
        found = true;
      }
      run = __shfl_sync(kFull, incl, 31);
    }
    total = run;
    if (lane == 0) s_item = total == (uint32_t)items ? item : (uint32_t)blockIdx.x;
  }
  __syncthreads();
  bwd_tile<FUSED, DEP, PPT, U8>(cfg, ws, a, (int64_t)s_item);
}

// Chain of the 2D adjoints through the projection, per Gaussian over all
// views; parameter gradients are added once per Gaussian (no atomics), pose
// partials are reduced per view across the CTA.
constexpr int kPoseSmemViews = 256;  // per-CTA pose sums in shared memory up to this many views

// The chain rule of one (view, Gaussian) entry: its 2D adjoints A0-A2 (mean,
// conic, opacity, depth, colour) through the projection of Sec. "3D Gaussian
// Splatting Representation" to the Gaussian's mean, scale, rotation, opacity
// and SH coefficients (added to g_* and, per coefficient q, through
// gsh_add(q, value), when PARAMS) and, when want_pose, to the view's six pose
// terms under the right perturbation T Exp(xi) (Eq. 3dgs_jacobi), written to
// pose[].  R0, R1: the entry's record (the conic the forward used); mu, s, Rg:
// the Gaussian's mean, scales and rotation; sh(k, ch): its SH coefficient k of
// colour channel ch.
template <int DEG, bool PARAMS, class ShAt, class ShGradAdd>
__device__ __forceinline__ void entry_chain(const Cam& cam, const gs_config& cfg, int width, int height,
                                            const float (&mu)[3], const float (&s)[3], const float (&Rg)[3][3],
                                            float4 R0, float4 R1, float4 A0, float4 A1, float4 A2, ShAt sh,
                                            ShGradAdd gsh_add, float (&g_mu)[3], float (&g_s)[3], float (&g_R)[3][3],
                                            float& g_o, bool want_pose, float* pose) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const float gmx = A0.x, gmy = A0.y, ga = A0.z, gb = A0.w, gc = A1.x, gop = A1.y, gdep = A1.z;
  const float gcol[3] = {A2.x, A2.y, A2.z};
  const float3 mh = to_camera(cam, mu[0], mu[1], mu[2]);
  const float iz = 1.f / mh.z;
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
  float U[3], Vv[3], rm0[3], rm1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    rm0[k] = Rg[0][k] * m0[0] + Rg[1][k] * m0[1] + Rg[2][k] * m0[2];
    rm1[k] = Rg[0][k] * m1[0] + Rg[1][k] * m1[1] + Rg[2][k] * m1[2];
    U[k] = s[k] * rm0[k];
    Vv[k] = s[k] * rm1[k];
  }
  // conic = Q = Sigma'^-1 from the stored record (the values the forward used)
  const float qa = R0.z, qb = R0.w, qc = R1.x;
  // dL/dSigma' = -Q G Q with G = [[ga, gb/2], [gb/2, gc]]
  const float hb = 0.5f * gb;
  const float P00 = qa * ga + qb * hb, P01 = qa * hb + qb * gc, P10 = qb * ga + qc * hb, P11 = qb * hb + qc * gc;
  const float gA = -(P00 * qa + P01 * qb);
  const float gBh = -(P00 * qb + P01 * qc);  // d/dSigma'_01 (one of the two symmetric entries)
  const float gCc = -(P10 * qb + P11 * qc);
  const float gB = 2.f * gBh;
  // A = U.U + dil, B = U.V, C = V.V + dil
  float gU[3], gV[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gU[k] = 2.f * gA * U[k] + gB * Vv[k];
    gV[k] = gB * U[k] + 2.f * gCc * Vv[k];
  }
  float gm0[3] = {0.f, 0.f, 0.f}, gm1[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (PARAMS) g_s[k] += gU[k] * rm0[k] + gV[k] * rm1[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (PARAMS) g_R[i][k] += s[k] * (gU[k] * m0[i] + gV[k] * m1[i]);
      gm0[i] += s[k] * gU[k] * Rg[i][k];
      gm1[i] += s[k] * gV[k] * Rg[i][k];
    }
  }
  // m0 = R^T J0, m1 = R^T J1  ->  dL/dJ0 = R gm0, dL/dJ1 = R gm1
  float gJ0[3], gJ1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gJ0[i] = cam.R[3 * i] * gm0[0] + cam.R[3 * i + 1] * gm0[1] + cam.R[3 * i + 2] * gm0[2];
    gJ1[i] = cam.R[3 * i] * gm1[0] + cam.R[3 * i + 1] * gm1[1] + cam.R[3 * i + 2] * gm1[2];
  }
  const float iz2 = iz * iz;
  float gx = gmx * cam.fx * iz, gy = gmy * cam.fy * iz;
  float gz = gdep - gmx * cam.fx * mh.x * iz2 - gmy * cam.fy * mh.y * iz2;
  gz += -gJ0[0] * cam.fx * iz2 - gJ1[1] * cam.fy * iz2;
  // J02 = -fx txc / z: unclamped txc = x/z, clamped txc constant
  gz += gJ0[2] * cam.fx * txc * iz2 * (clx ? 1.f : 2.f);
  if (!clx) gx += -gJ0[2] * cam.fx * iz2;
  gz += gJ1[2] * cam.fy * tyc * iz2 * (cly ? 1.f : 2.f);
  if (!cly) gy += -gJ1[2] * cam.fy * iz2;
  // dL/dmu through mu_hat = R mu + t
  float gWm[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) gWm[j] = cam.R[j] * gx + cam.R[3 + j] * gy + cam.R[6 + j] * gz;
  // colour: raw = sum_k SH_k Y_k(dir) + 0.5, clamped at 0
  const float3 cw = camera_centre(cam);
  float dv[3] = {mu[0] - cw.x, mu[1] - cw.y, mu[2] - cw.z};
  const float inv = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const float dx = dv[0] * inv, dy = dv[1] * inv, dz = dv[2] * inv;
  float Y[16];
  sh_basis<DEG>(dx, dy, dz, Y);
  float graw[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float raw = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) raw += sh(k, ch) * Y[k];
    graw[ch] = raw > 0.f ? gcol[ch] : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (PARAMS) gsh_add(3 * k + ch, graw[ch] * Y[k]);
  }
  // d colour / d dir = sum_k (sum_ch graw_ch SH_k,ch) grad Y_k
  float wk[16];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    wk[k] = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) wk[k] += graw[ch] * sh(k, ch);
  }
  const float3 gd3 = sh_weighted_grad<DEG>(wk, dx, dy, dz);
  const float gdir[3] = {gd3.x, gd3.y, gd3.z};
  const float dd = dx * gdir[0] + dy * gdir[1] + dz * gdir[2];
  const float gv[3] = {(gdir[0] - dx * dd) * inv, (gdir[1] - dy * dd) * inv, (gdir[2] - dz * dd) * inv};
#pragma unroll
  for (int j = 0; j < 3; ++j)
    if (PARAMS) g_mu[j] += gWm[j] + gv[j];
  if (PARAMS) g_o += gop;
  if (want_pose) {
    // right perturbation T Exp(xi), xi = (rho, theta):
    //   d mu_hat = R rho + R (theta x mu), d m = m x theta, d c_w = -rho + c_w x theta
    const float gcw[3] = {-gv[0], -gv[1], -gv[2]};
    pose[0] = gWm[0] - gcw[0];
    pose[1] = gWm[1] - gcw[1];
    pose[2] = gWm[2] - gcw[2];
    // theta: mu x (R^T g_mu_hat) + gm0 x m0 + gm1 x m1 + g_cw x c_w
    const float c_w[3] = {cw.x, cw.y, cw.z};
    pose[3] = mu[1] * gWm[2] - mu[2] * gWm[1] + gm0[1] * m0[2] - gm0[2] * m0[1] + gm1[1] * m1[2] -
              gm1[2] * m1[1] + gcw[1] * c_w[2] - gcw[2] * c_w[1];
    pose[4] = mu[2] * gWm[0] - mu[0] * gWm[2] + gm0[2] * m0[0] - gm0[0] * m0[2] + gm1[2] * m1[0] -
              gm1[0] * m1[2] + gcw[2] * c_w[0] - gcw[0] * c_w[2];
    pose[5] = mu[0] * gWm[1] - mu[1] * gWm[0] + gm0[0] * m0[1] - gm0[1] * m0[0] + gm1[0] * m1[1] -
              gm1[1] * m1[0] + gcw[0] * c_w[1] - gcw[1] * c_w[0];
  }
}

// PARAMS: parameter gradients are wanted; without them (the pose gradient
// alone, the map held fixed) their accumulation is left out at compile time.
template <int DEG, bool BF16, bool PARAMS>
__global__ void __launch_bounds__(256, 2) k_preprocess_bwd(gs_map map, const gs_camera* __restrict__ cams,
                                                        gs_config cfg, Ws ws, BwdArgs a) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  // SH gradient accumulators and the Gaussian's SH coefficients live in
  // shared memory (one column per thread): coefficients are fetched once, with
  // independent coalesced loads, and reused by every view
  // (dynamic shared memory: 3K * 256 floats each, up to 48 KB; the gradient
  // columns only when parameter gradients are wanted)
  extern __shared__ float s_dyn[];
  float(*s_gsh)[256] = reinterpret_cast<float(*)[256]>(s_dyn);
  float(*s_sh)[256] = reinterpret_cast<float(*)[256]>(s_dyn + (PARAMS ? 3 * K * 256 : 0));
  // per-view pose sums of the CTA (6 V floats after the SH columns), added to
  // the global pose gradient once per CTA; with more views, global atomics
  float* s_pose = s_dyn + (PARAMS ? 2 : 1) * 3 * K * 256;
  const int64_t n = ws.n;
  if (ws.counters[kStatus] != 0) return;
  // one thread per Gaussian of the list of those seen by some view, so that
  // warps are full although most of the map is outside every view
  const uint32_t count = ws.counters[kGaussCount];
  if ((uint64_t)blockIdx.x * blockDim.x >= count) return;  // the whole CTA
  const uint64_t li = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool any = li < count;
  const int64_t g = any ? (int64_t)ws.gauss_list[li] : 0;
  const bool in_range = any;
  const bool want_pose = a.grad_pose != nullptr;
  if (!want_pose && !__any_sync(kFull, any)) return;
  const bool pose_smem = want_pose && ws.views <= kPoseSmemViews;
  if (pose_smem) {  // every warp of the CTA is here (the early return above needs !want_pose)
    for (int i = threadIdx.x; i < 6 * ws.views; i += blockDim.x) s_pose[i] = 0.f;
    __syncthreads();
  }

  float mu[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f}, logit = 0.f;
  if (any) {
    mu[0] = map.mean[g]; mu[1] = map.mean[n + g]; mu[2] = map.mean[2 * n + g];
    ls[0] = map.log_scale[g]; ls[1] = map.log_scale[n + g]; ls[2] = map.log_scale[2 * n + g];
    q[0] = map.quat[g]; q[1] = map.quat[n + g]; q[2] = map.quat[2 * n + g]; q[3] = map.quat[3 * n + g];
    logit = map.logit_opacity[g];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) s_sh[3 * k + ch][threadIdx.x] = sh_coeff<BF16>(map.sh_dc, map.sh_rest, n, g, k, ch);
  }
  const float qi = rsqrtf(fmaxf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3], 1e-30f));
  const float qw = q[0] * qi, qx = q[1] * qi, qy = q[2] * qi, qz = q[3] * qi;
  float Rg[3][3];
  quat_to_rot(qw, qx, qy, qz, Rg);
  float s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = expf(ls[k]);
  const float o = 1.f / (1.f + expf(-logit));

  float g_mu[3] = {0.f, 0.f, 0.f}, g_s[3] = {0.f, 0.f, 0.f}, g_R[3][3] = {{0.f}}, g_o = 0.f;
#pragma unroll
  for (int k = 0; k < 3 * K; ++k)
    if (PARAMS) s_gsh[k][threadIdx.x] = 0.f;

  // The per-(Gaussian, view) chain rule; pose[] receives this view's
  // contribution to the pose gradient.
  auto view_bwd = [&](const int v, float pose[6]) {
    const int64_t e = (int64_t)v * n + g;
    float4* ad = ws.adjoints + 3 * e;
    entry_chain<DEG, PARAMS>(
        load_cam(cams, v), cfg, ws.width, ws.height, mu, s, Rg, ws.records[3 * e], ws.records[3 * e + 1], ad[0],
        ad[1], ad[2], [&](int k, int ch) { return s_sh[3 * k + ch][threadIdx.x]; },
        [&](int q, float val) { s_gsh[q][threadIdx.x] += val; }, g_mu, g_s, g_R, g_o, want_pose, pose);
    // consume: leave the adjoint area zero for the next backward of this projection
    ad[0] = ad[1] = ad[2] = make_float4(0.f, 0.f, 0.f, 0.f);
  };
  // Views are taken 32 at a time.  Each lane collects the views in which its
  // Gaussian has a non-empty box.  When those sets are much alike across the
  // warp, the views are taken in turn by all lanes together and the pose sums
  // are warp reductions; otherwise each lane runs over its own views only (so
  // that lanes are not left idle when the Gaussians are outside most views)
  // and adds its pose terms one by one.
  for (int v0 = 0; v0 < ws.views; v0 += 32) {
    const int nv = min(32, ws.views - v0);
    uint32_t vis_mask = 0;
    if (in_range)
      for (int j = 0; j < nv; ++j)
        if (!rect_empty(ws.rects[(int64_t)(v0 + j) * n + g])) vis_mask |= 1u << j;
    const uint32_t warp_mask = __reduce_or_sync(kFull, vis_mask);
    const uint32_t most = __reduce_max_sync(kFull, (uint32_t)__popc(vis_mask));
    if ((uint32_t)__popc(warp_mask) <= most + 1) {
      for (uint32_t mk = warp_mask; mk; mk &= mk - 1) {
        const int v = v0 + __ffs(mk) - 1;
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if ((vis_mask >> (v - v0)) & 1u) view_bwd(v, pose);
        if (want_pose) {
#pragma unroll
          for (int k = 0; k < 6; ++k) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) pose[k] += __shfl_xor_sync(kFull, pose[k], off);
          }
          if ((threadIdx.x & 31) == 0) {
            float* dst = (pose_smem ? s_pose : a.grad_pose) + 6 * v;
#pragma unroll
            for (int k = 0; k < 6; ++k)
              if (pose[k] != 0.f) atomicAdd(dst + k, pose[k]);
          }
        }
      }
    } else {
      while (vis_mask) {
        const int v = v0 + __ffs(vis_mask) - 1;
        vis_mask &= vis_mask - 1;
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        view_bwd(v, pose);
        if (want_pose) {
          float* dst = (pose_smem ? s_pose : a.grad_pose) + 6 * v;
#pragma unroll
          for (int k = 0; k < 6; ++k) atomicAdd(dst + k, pose[k]);
        }
      }
    }
  }
  if (pose_smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < 6 * ws.views; i += blockDim.x)
      if (s_pose[i] != 0.f) atomicAdd(a.grad_pose + i, s_pose[i]);
  }
  if (!PARAMS || !any) return;  // no parameter gradients wanted: pose only
  // quaternion: R(q^) entries -> q^ -> q (normalisation)
  const float gw = 2.f * (-qz * g_R[0][1] + qy * g_R[0][2] + qz * g_R[1][0] - qx * g_R[1][2] - qy * g_R[2][0] +
                          qx * g_R[2][1]);
  const float gxq = 2.f * (qy * g_R[0][1] + qz * g_R[0][2] + qy * g_R[1][0] - 2.f * qx * g_R[1][1] - qw * g_R[1][2] +
                           qz * g_R[2][0] + qw * g_R[2][1] - 2.f * qx * g_R[2][2]);
  const float gyq = 2.f * (-2.f * qy * g_R[0][0] + qx * g_R[0][1] + qw * g_R[0][2] + qx * g_R[1][0] + qz * g_R[1][2] -
                           qw * g_R[2][0] + qz * g_R[2][1] - 2.f * qy * g_R[2][2]);
  const float gzq = 2.f * (-2.f * qz * g_R[0][0] - qw * g_R[0][1] + qx * g_R[0][2] + qw * g_R[1][0] -
                           2.f * qz * g_R[1][1] + qy * g_R[1][2] + qx * g_R[2][0] + qy * g_R[2][1]);
  const float dq = qw * gw + qx * gxq + qy * gyq + qz * gzq;
  // Add to the caller's gradients.  The loads of a group are issued before
  // any of its stores: the gradient arrays may alias as far as the compiler
  // knows, so interleaved read-modify-writes would serialise on memory latency.
  {
    float* dst[11] = {a.grad_quat + g,         a.grad_quat + n + g,     a.grad_quat + 2 * n + g,
                      a.grad_quat + 3 * n + g, a.grad_mean + g,         a.grad_mean + n + g,
                      a.grad_mean + 2 * n + g, a.grad_log_scale + g,    a.grad_log_scale + n + g,
                      a.grad_log_scale + 2 * n + g, a.grad_logit + g};
    const float add[11] = {(gw - qw * dq) * qi, (gxq - qx * dq) * qi, (gyq - qy * dq) * qi, (gzq - qz * dq) * qi,
                           g_mu[0], g_mu[1], g_mu[2], g_s[0] * s[0], g_s[1] * s[1], g_s[2] * s[2],
                           g_o * o * (1.f - o)};
    float cur[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) cur[i] = *dst[i];
#pragma unroll
    for (int i = 0; i < 11; ++i) *dst[i] = cur[i] + add[i];
  }
  constexpr int kGroup = 8;
#pragma unroll
  for (int q0 = 0; q0 < 3 * K; q0 += kGroup) {
    float cur[kGroup];
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
      const int q = q0 + i;
      if (q < 3 * K) cur[i] = q < 3 ? a.grad_sh_dc[q * n + g] : a.grad_sh_rest[(int64_t)(q - 3) * n + g];
    }
#pragma unroll
    for (int i = 0; i < kGroup; ++i) {
      const int q = q0 + i;
      if (q >= 3 * K) continue;
      const float v = cur[i] + s_gsh[q][threadIdx.x];
      if (q < 3) a.grad_sh_dc[q * n + g] = v;
      else a.grad_sh_rest[(int64_t)(q - 3) * n + g] = v;
    }
  }
}

// Pose-only projection backward (the map held fixed, e.g. camera tracking):
// one thread per visible (view, Gaussian) entry, in the projection's order of
// the entries (ws.visible).  That order holds, per warp of the projection, the
// entries of 32 consecutive Gaussians view by view, so neighbouring threads
// gather the parameters, records and adjoints of neighbouring Gaussians, and
// every thread has one entry's work.  (A thread per Gaussian walks the views
// that see it, which differ from lane to lane when the cameras sit inside the
// map; the depth-sorted order scatters the gathers.)  A warp sums its
// entries' pose terms over each run of one view with a segmented shuffle
// reduction; the run's first lane adds the sums to the CTA's per-view sums in
// shared memory (to grad_pose directly beyond kPoseSmemViews views), which
// are added to grad_pose once per CTA.
constexpr int kPoseEntryThreads = 256;

template <int DEG, bool BF16>
__global__ void __launch_bounds__(kPoseEntryThreads) k_pose_bwd_entries(gs_map map, const gs_camera* __restrict__ cams,
                                                                      gs_config cfg, Ws ws, BwdArgs a) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ float s_pose[6 * kPoseSmemViews];
  if (ws.counters[kStatus] != 0) return;
  const int64_t n = ws.n;
  const uint32_t nvis = ws.counters[kVisibleCount];
  const uint32_t per = ((nvis + gridDim.x - 1) / gridDim.x + kPoseEntryThreads - 1) / kPoseEntryThreads *
                       kPoseEntryThreads;
  const uint64_t i0 = (uint64_t)blockIdx.x * per;
  if (i0 >= nvis) return;  // the whole CTA
  const uint64_t i1 = min((uint64_t)nvis, i0 + per);
  const bool want_pose = a.grad_pose != nullptr;
  const bool pose_smem = ws.views <= kPoseSmemViews;
  if (pose_smem)
    for (int i = threadIdx.x; i < 6 * ws.views; i += kPoseEntryThreads) s_pose[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (uint64_t b = i0; b < i1; b += kPoseEntryThreads) {
    const uint64_t i = b + threadIdx.x;
    const bool act = i < i1;
    const uint32_t e = ws.visible[act ? i : i0];
    const int v = (int)(e / (uint64_t)n);
    const int64_t g = (int64_t)e - (int64_t)v * n;
    float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (act) {
      const float mu[3] = {map.mean[g], map.mean[n + g], map.mean[2 * n + g]};
      const float q[4] = {map.quat[g], map.quat[n + g], map.quat[2 * n + g], map.quat[3 * n + g]};
      float s[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) s[k] = expf(map.log_scale[k * n + g]);
      const float qi = rsqrtf(fmaxf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3], 1e-30f));
      float Rg[3][3];
      quat_to_rot(q[0] * qi, q[1] * qi, q[2] * qi, q[3] * qi, Rg);
      float sh[3 * K];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) sh[3 * k + ch] = sh_coeff<BF16>(map.sh_dc, map.sh_rest, n, g, k, ch);
      float g_mu[3], g_s[3], g_R[3][3], g_o;  // parameter sums: not formed without PARAMS
      float4* ad = ws.adjoints + 3 * (int64_t)e;
      entry_chain<DEG, false>(
          load_cam(cams, v), cfg, ws.width, ws.height, mu, s, Rg, ws.records[3 * (int64_t)e],
          ws.records[3 * (int64_t)e + 1], ad[0], ad[1], ad[2], [&](int k, int ch) { return sh[3 * k + ch]; },
          [](int, float) {}, g_mu, g_s, g_R, g_o, want_pose, pose);
      // consume: leave the adjoint area zero for the next backward of this projection
      ad[0] = ad[1] = ad[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!want_pose) continue;
    // runs of one view among the warp's lanes: lane l's run ends at the first
    // lane j >= l whose next lane holds another view (or j = 31)
    const int vn = __shfl_down_sync(kFull, v, 1);
    const unsigned ends = __ballot_sync(kFull, lane == 31 || vn != v);
    const int last = __ffs(ends & ~((1u << lane) - 1u)) - 1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const float y = __shfl_down_sync(kFull, pose[k], d);
        if (lane + d <= last) pose[k] += y;
      }
    const bool head = lane == 0 || ((ends >> (lane - 1)) & 1u);
    if (head)
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (pose[k] != 0.f) atomicAdd((pose_smem ? s_pose : a.grad_pose) + 6 * v + k, pose[k]);
  }
  __syncthreads();
  if (!want_pose || !pose_smem) return;
  for (int i = threadIdx.x; i < 6 * ws.views; i += kPoseEntryThreads)
    if (s_pose[i] != 0.f) atomicAdd(a.grad_pose + i, s_pose[i]);
}

template <int DEG, bool BF16>
static cudaError_t launch_pose_bwd_entries(const gs_map& map, const gs_camera* cams, const gs_config& cfg,
                                           const Ws& ws, const BwdArgs& a, cudaStream_t st) {
  trace_begin(kKPreprocessBwd, st);
  k_pose_bwd_entries<DEG, BF16><<<(unsigned)sm_count() * 4, kPoseEntryThreads, 0, st>>>(map, cams, cfg, ws, a);
  trace_end(st);
  return cudaGetLastError();
}

template <int DEG, bool BF16, bool PARAMS>
static cudaError_t launch_pre_bwd_t(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                    const BwdArgs& a, cudaStream_t st) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const size_t smem =
      ((size_t)(PARAMS ? 2 : 1) * 3 * K * 256 + (ws.views <= kPoseSmemViews ? 6 * ws.views : 0)) * sizeof(float);
  cudaError_t err = cudaFuncSetAttribute(k_preprocess_bwd<DEG, BF16, PARAMS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  trace_begin(kKPreprocessBwd, st);
  k_preprocess_bwd<DEG, BF16, PARAMS><<<(unsigned)((ws.n + 255) / 256), 256, smem, st>>>(map, cams, cfg, ws, a);
  trace_end(st);
  return cudaGetLastError();
}

template <int DEG, bool BF16>
static cudaError_t launch_pre_bwd(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                  const BwdArgs& a, cudaStream_t st) {
  return a.grad_mean ? launch_pre_bwd_t<DEG, BF16, true>(map, cams, cfg, ws, a, st)
                     : launch_pose_bwd_entries<DEG, BF16>(map, cams, cfg, ws, a, st);
}

cudaError_t launch_bwd_prologue(const Ws& ws, const BwdArgs& a, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(ws.view_stats, 0, (size_t)ws.views * 4 * sizeof(float), st);
  if (err != cudaSuccess) return err;
  const bool fused = a.fused();
  const int64_t hw = (int64_t)ws.width * ws.height;
  if (fused && a.tgt_depth && a.w_depth != 0.f) {
    const int64_t nblk = (hw + 255) / 256;
    dim3 grid((unsigned)(nblk < 1024 ? nblk : 1024), (unsigned)ws.views);
    trace_begin(kKCountDepth, st);
    k_count_depth<<<grid, 256, 0, st>>>(a.tgt_depth, hw, ws.view_stats);
    trace_end(st);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

cudaError_t launch_preprocess_bwd(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                  const BwdArgs& a, cudaStream_t st) {
  const bool bf = map.sh_bf16 != 0;
  switch (map.sh_degree) {
    case 0: return bf ? launch_pre_bwd<0, true>(map, cams, cfg, ws, a, st) : launch_pre_bwd<0, false>(map, cams, cfg, ws, a, st);
    case 1: return bf ? launch_pre_bwd<1, true>(map, cams, cfg, ws, a, st) : launch_pre_bwd<1, false>(map, cams, cfg, ws, a, st);
    case 2: return bf ? launch_pre_bwd<2, true>(map, cams, cfg, ws, a, st) : launch_pre_bwd<2, false>(map, cams, cfg, ws, a, st);
    default: return bf ? launch_pre_bwd<3, true>(map, cams, cfg, ws, a, st) : launch_pre_bwd<3, false>(map, cams, cfg, ws, a, st);
  }
}

// One CTA per work item; the hardware starts them in index order, which is
// the work list's longest-first order.
template <bool FUSED, bool DEP, bool U8 = false>
static cudaError_t launch_blend_bwd(const gs_config& cfg, const Ws& ws, const BwdArgs& a, int64_t items,
                                    cudaStream_t st) {
  if (items < 1) return cudaSuccess;
  k_render_bwd<FUSED, DEP, kBwdPPT, U8><<<(unsigned)items, 256 / kBwdPPT, 0, st>>>(cfg, ws, a);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                              const BwdArgs& a, cudaStream_t st) {
  const bool fused = a.fused();
  const int64_t items = (int64_t)ws.views * ws.tiles_per_view;
  const bool dep = (fused && a.tgt_depth && a.w_depth != 0.f) || a.dl_ddepth || a.dl_dopac;
  // per-view loss accumulators and valid-depth counts, then the work-list fill counts (adjacent in the layout)
  const size_t cleared = (size_t)(reinterpret_cast<char*>(ws.work_fill + kWorkClasses) -
                                  reinterpret_cast<char*>(ws.view_stats));
  cudaError_t err = cudaMemsetAsync(ws.view_stats, 0, cleared, st);
  if (err != cudaSuccess) return err;
  const float* depth_count = fused && a.tgt_depth && a.w_depth != 0.f ? a.tgt_depth : nullptr;
  trace_begin(kKTileWork, st);
  k_tile_work<<<(unsigned)((items + kWorkItemsPerCta - 1) / kWorkItemsPerCta), kWorkThreads, 0, st>>>(
      ws, a.n_contrib, depth_count);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  trace_begin(kKRenderBwd, st);
  if (fused && a.tgt_rgb8) {
    if (dep) err = launch_blend_bwd<true, true, true>(cfg, ws, a, items, st);
    else err = launch_blend_bwd<true, false, true>(cfg, ws, a, items, st);
  } else if (fused) {
    if (dep) err = launch_blend_bwd<true, true>(cfg, ws, a, items, st);
    else err = launch_blend_bwd<true, false>(cfg, ws, a, items, st);
  } else {
    if (dep) err = launch_blend_bwd<false, true>(cfg, ws, a, items, st);
    else err = launch_blend_bwd<false, false>(cfg, ws, a, items, st);
  }
  trace_end(st);
  if (err != cudaSuccess) return err;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_preprocess_bwd(map, cams, cfg, ws, a, st);
}

}  // namespace gsb
