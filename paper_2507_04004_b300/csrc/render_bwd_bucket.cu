// Per-Gaussian backward of the blending (arxiv 2507.04004, Sec. "Per-Gaussian
// Backpropagation", Fig. cuda (b1), (b2)), an alternative to the
// pixel-parallel blend backward of render_bwd.cu with the same outputs (the
// per-(view, Gaussian) 2D adjoints in the workspace, then the shared
// projection backward).
//
// The depth-sorted Gaussians of a tile are cut into buckets of 32.  One warp
// owns a bucket, each lane one of its Gaussians, and the tile's pixels stream
// through the lanes in pixel order: lane j handles pixel number q at step
// q + j, right after lane j - 1 handled it, and receives from it (one shuffle
// each) the pixel's transmittance T and its adjoint-weighted output in front of
// Gaussian j.  A lane sums its Gaussian's adjoints over the pixels in
// registers and adds them to the workspace once per (Gaussian, tile), so
// pixels never collide on an atomic.  The state at the start of a bucket is
// the forward's checkpoint; only pixels whose contributors reach into the
// bucket are streamed.
//
// Per pixel, with the adjoint a = (dL/dC_r, dL/dC_g, dL/dC_b, dL/dD, dL/dO)
// and f_i = (c_i, d_i, 1) for Gaussian i, the rendered output is
// Y = sum_i f_i alpha_i T_i (plus the background T_final in colour), and with
// A_i = a . sum_{j <= i} f_j alpha_j T_j the adjoint of alpha_i is
//   dL/dalpha_i = T_i a.f_i - (a.Y - A_i) / (1 - alpha_i),
// the second term being the part of the output behind Gaussian i.
#include "gs_internal.h"

namespace gsb {

constexpr int kBkWarps = 4;  // warps (buckets in flight) per tile

size_t bucket_ws_bytes(const Ws& ws) {
  const int64_t tiles = (int64_t)ws.views * ws.tiles_per_view;
  const int64_t nbuckets = ws.cap / 32 + tiles + 1;
  const size_t pix = ((size_t)tiles * 8 * 256 * sizeof(float) + 255) / 256 * 256;
  return pix + (size_t)nbuckets * 5 * 256 * sizeof(float);
}

BucketWs resolve_bucket_ws(const Ws& ws, void* ptr) {
  const int64_t tiles = (int64_t)ws.views * ws.tiles_per_view;
  const size_t pix = ((size_t)tiles * 8 * 256 * sizeof(float) + 255) / 256 * 256;
  BucketWs b;
  b.pix = static_cast<float*>(ptr);
  b.ckpt = reinterpret_cast<float*>(static_cast<char*>(ptr) + pix);
  b.nbuckets = ws.cap / 32 + tiles + 1;
  return b;
}

// Per-pixel adjoints (the fused loss of Eq. depth_loss and/or the caller's),
// the adjoint-weighted output a.Y and the contributor count, tile-major.
template <bool FUSED>
__global__ void __launch_bounds__(256) k_pixel_adjoint(gs_config cfg, Ws ws, BwdArgs a, BucketWs bw) {
  __shared__ float s_red[8];
  if (ws.counters[kStatus] != 0) return;
  const int64_t tile = blockIdx.x;
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int lp = threadIdx.x;
  const int x = (t % ws.tiles_x) * kTile + (lp & 15), y = (t / ws.tiles_x) * kTile + (lp >> 4);
  const int64_t HW = (int64_t)ws.width * ws.height;
  const uint32_t cnt = ws.tile_count[tile];
  float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float ay = 0.f, loss = 0.f;
  uint32_t nc = 0;
  if (x < ws.width && y < ws.height) {
    const int64_t p = (int64_t)y * ws.width + x;
    nc = min(a.n_contrib[v * HW + p], cnt);
    const float C[3] = {a.rgb[(3 * (int64_t)v + 0) * HW + p], a.rgb[(3 * (int64_t)v + 1) * HW + p],
                        a.rgb[(3 * (int64_t)v + 2) * HW + p]};
    const float Dp = a.depth[v * HW + p];
    const float Tf = a.t_final[v * HW + p];
    if (FUSED) {
      const float inv3hw = a.w_rgb / (3.f * (float)HW);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float r = C[ch] - a.tgt_rgb[(3 * (int64_t)v + ch) * HW + p];
        g[ch] = inv3hw * (float)((r > 0.f) - (r < 0.f));
        loss += inv3hw * fabsf(r);
      }
      if (a.tgt_depth && a.w_depth != 0.f) {
        const float ds = a.tgt_depth[v * HW + p];
        const float O = a.opac[v * HW + p];
        const float nd = ws.view_stats[4 * v + 1];
        if (ds > 0.f && O > 0.f && nd > 0.f) {
          const float rd = Dp / O - ds;
          const float sg = (float)((rd > 0.f) - (rd < 0.f));
          g[3] = a.w_depth * sg / (O * nd);
          g[4] = -a.w_depth * sg * Dp / (O * O * nd);
          loss += a.w_depth * fabsf(rd) / nd;
        }
      }
    }
    if (a.dl_drgb)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g[ch] += a.dl_drgb[(3 * (int64_t)v + ch) * HW + p];
    if (a.dl_ddepth) g[3] += a.dl_ddepth[v * HW + p];
    if (a.dl_dopac) g[4] += a.dl_dopac[v * HW + p];
    ay = g[0] * C[0] + g[1] * C[1] + g[2] * C[2] + g[3] * Dp + g[4] * (1.f - Tf);
  }
  float* out = bw.pix + tile * (8 * 256);
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q * 256 + lp] = g[q];
  out[5 * 256 + lp] = ay;
  out[6 * 256 + lp] = __uint_as_float(nc);
  if (FUSED && a.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(kFull, loss, o);
    if ((lp & 31) == 0) s_red[lp >> 5] = loss;
    __syncthreads();
    if (lp == 0) {
      float tot = 0.f;
      for (int i = 0; i < 8; ++i) tot += s_red[i];
      if (tot != 0.f) atomicAdd(a.loss + v, tot);
    }
  }
}

__global__ void __launch_bounds__(32 * kBkWarps) k_render_bwd_bucket(gs_config cfg, Ws ws, BucketWs bw) {
  __shared__ float4 s_a[256];                  // dL/dC_r, dL/dC_g, dL/dC_b, dL/dD
  __shared__ float2 s_b[256];                  // dL/dO, a.Y
  __shared__ uint32_t s_nc[256];
  __shared__ uint32_t s_list[kBkWarps][256];   // streamed pixels: index | min(32, n_contrib - bucket start) << 8
  __shared__ float2 s_ck[kBkWarps][32];        // (T, A) at the bucket start of 32 streamed pixels
  __shared__ uint32_t s_max;
  if (ws.counters[kStatus] != 0) return;
  const int64_t tile = blockIdx.x;
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t start = ws.tile_start[tile], cnt = ws.tile_count[tile];
  const float* pix = bw.pix + tile * (8 * 256);
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  uint32_t mx = 0;
  for (int i = threadIdx.x; i < 256; i += 32 * kBkWarps) {
    s_a[i] = make_float4(pix[i], pix[256 + i], pix[512 + i], pix[768 + i]);
    s_b[i] = make_float2(pix[1024 + i], pix[1280 + i]);
    const uint32_t nc = __float_as_uint(pix[1536 + i]);
    s_nc[i] = nc;
    mx = max(mx, nc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane == 0) atomicMax(&s_max, mx);
  __syncthreads();
  const uint32_t maxnc = min(s_max, cnt);
  const int nbk = (int)((maxnc + 31u) >> 5);
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  float4* adj = ws.adjoints + 3 * (int64_t)v * ws.n;
  const float a_max = cfg.alpha_max;
  const float lt = __log2f(cfg.alpha_min);
  const float ox = (float)((t % ws.tiles_x) * kTile) + 0.5f, oy = (float)((t / ws.tiles_x) * kTile) + 0.5f;
  uint32_t* list = s_list[warp];
  float2* ring = s_ck[warp];

  for (int k = warp; k < nbk; k += kBkWarps) {
    const uint32_t ig = 32u * (uint32_t)k + (uint32_t)lane;  // this lane's Gaussian: its place in the tile list
    const bool g_ok = ig < maxnc;
    uint32_t gid = 0;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, c = g0;
    if (g_ok) {
      gid = ws.sorted_ids[start + ig];
      const float4* r = rec + 3 * (int64_t)gid;
      const Staged sg = stage_gaussian(r[0], r[1]);
      g0 = sg.g0;
      g1 = sg.g1;
      c = r[2];
    }
    // the pixels whose contributors reach into this bucket, in pixel order
    __syncwarp();
    uint32_t m = 0;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int p = 32 * c8 + lane;
      const uint32_t nc = s_nc[p];
      const bool in = nc > 32u * (uint32_t)k;
      const unsigned b = __ballot_sync(kFull, in);
      if (in) list[m + __popc(b & ((1u << lane) - 1u))] = (uint32_t)p | (min(nc - 32u * (uint32_t)k, 32u) << 8);
      m += (uint32_t)__popc(b);
    }
    __syncwarp();
    const float* ck = bw.ckpt + ((int64_t)(start >> 5) + tile + k) * (5 * 256);
    // checkpoints of the streamed pixels, fetched one chunk of 32 ahead
    float pre[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int pre_p = -1;
    if ((uint32_t)lane < m) {
      pre_p = (int)(list[lane] & 255u);
#pragma unroll
      for (int q = 0; q < 5; ++q) pre[q] = ck[q * 256 + pre_p];
    }
    // sums over the pixels: dp dx, dp dy, dp dx^2, dp dx dy, dp dy^2, dp (dp = dL/dpower,
    // zero where alpha is clamped), and dL/dD w, dL/dC w (w = alpha T)
    float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 0.f, v6 = 0.f, v7 = 0.f, v8 = 0.f, v9 = 0.f;
    float Tst = 0.f, Ast = 0.f;
    const uint32_t steps = m + 31u;
    for (uint32_t s = 0; s < steps; ++s) {
      if ((s & 31u) == 0) {
        __syncwarp();
        if (pre_p >= 0) {
          const float4 a4 = s_a[pre_p];
          const float2 b2 = s_b[pre_p];
          const float A0 = a4.x * pre[1] + a4.y * pre[2] + a4.z * pre[3] + a4.w * pre[4] + b2.x * (1.f - pre[0]);
          ring[lane] = make_float2(pre[0], A0);
        }
        __syncwarp();
        pre_p = -1;
        const uint32_t nxt = s + 32u + (uint32_t)lane;
        if (nxt < m) {
          pre_p = (int)(list[nxt] & 255u);
#pragma unroll
          for (int q = 0; q < 5; ++q) pre[q] = ck[q * 256 + pre_p];
        }
      }
      const float Tin = __shfl_up_sync(kFull, Tst, 1), Ain = __shfl_up_sync(kFull, Ast, 1);
      const int q = (int)s - lane;
      if (q >= 0 && q < (int)m) {
        float T = Tin, A = Ain;
        if (lane == 0) {
          const float2 c2 = ring[q & 31];
          T = c2.x;
          A = c2.y;
        }
        const uint32_t ent = list[q];
        const uint32_t p = ent & 255u, reach = ent >> 8;  // lanes below reach are in front of its last contributor
        const float px = ox + (float)(p & 15u), py = oy + (float)(p >> 4);
        const float p2 = blend_p2(g0, g1, px, py);
        if (g_ok && (uint32_t)lane < reach && p2 >= lt) {
          const float e = ex2_approx(p2);
          const float al = fminf(a_max, e);
          const float4 a4 = s_a[p];
          const float2 b2 = s_b[p];
          const float wg = fmaf(a4.x, c.x, fmaf(a4.y, c.y, fmaf(a4.z, c.z, fmaf(a4.w, g1.z, b2.x))));
          const float aT = al * T;
          A = fmaf(aT, wg, A);
          const float dA = T * wg - (b2.y - A) * __fdividef(1.f, 1.f - al);
          T = T * (1.f - al);
          const float dp = e > a_max ? 0.f : dA * al;
          const float dx = px - g0.x, dy = py - g0.y;
          const float dpx = dp * dx, dpy = dp * dy;
          q0 += dpx;
          q1 += dpy;
          q2 = fmaf(dpx, dx, q2);
          q3 = fmaf(dpx, dy, q3);
          q4 = fmaf(dpy, dy, q4);
          q5 += dp;
          v6 = fmaf(a4.w, aT, v6);
          v7 = fmaf(a4.x, aT, v7);
          v8 = fmaf(a4.y, aT, v8);
          v9 = fmaf(a4.z, aT, v9);
        }
        Tst = T;
        Ast = A;
      }
    }
    if (g_ok) {
      // the same 2D adjoints as the pixel-parallel kernel's flush
      const float gmx = -kLn2 * (2.f * g0.z * q0 + g0.w * q1);
      const float gmy = -kLn2 * (g0.w * q0 + 2.f * g1.x * q1);
      const float ga = -0.5f * q2, gb = -q3, gc = -0.5f * q4, go = q5 * g1.w;
      float4* dst = adj + 3 * (int64_t)gid;
      if (q0 != 0.f || q1 != 0.f || q2 != 0.f || q3 != 0.f) atomicAdd(dst, make_float4(gmx, gmy, ga, gb));
      if (q4 != 0.f || q5 != 0.f || v6 != 0.f) atomicAdd(dst + 1, make_float4(gc, go, v6, 0.f));
      if (v7 != 0.f || v8 != 0.f || v9 != 0.f) atomicAdd(dst + 2, make_float4(v7, v8, v9, 0.f));
    }
  }
}

cudaError_t launch_render_bwd_bucket(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                     const BwdArgs& a, const BucketWs& bw, cudaStream_t st) {
  cudaError_t err = launch_bwd_prologue(ws, a, st);
  if (err != cudaSuccess) return err;
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKPixelAdjoint, st);
  if (a.tgt_rgb) k_pixel_adjoint<true><<<ntiles, 256, 0, st>>>(cfg, ws, a, bw);
  else k_pixel_adjoint<false><<<ntiles, 256, 0, st>>>(cfg, ws, a, bw);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  trace_begin(kKRenderBwdBucket, st);
  k_render_bwd_bucket<<<ntiles, 32 * kBkWarps, 0, st>>>(cfg, ws, bw);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_preprocess_bwd(map, cams, cfg, ws, a, st);
}

}  // namespace gsb
