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
// bucket are streamed, as vertical pixel pairs through packed FP32 pairs.
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
  return (size_t)(ws.cap / 32 + tiles + 1) * 5 * 256 * sizeof(float);
}

BucketWs resolve_bucket_ws(const Ws& ws, void* ptr) {
  (void)ws;
  BucketWs b;
  b.ckpt = static_cast<float*>(ptr);
  return b;
}

// One CTA per (view, tile).  Staging: the pixel adjoints (the fused loss of
// Eq. depth_loss and/or the caller's), a.Y and the contributor counts of the
// tile's 256 pixels go to shared memory, stored by vertical pixel pair (rows
// 2r and 2r + 1 of one column) so that one 16-byte load gives a packed FP32
// pair of two values.  Then each warp takes buckets of the tile in turn and
// streams the pairs that reach into the bucket, one pair per lane and step.
template <bool FUSED>
__global__ void __launch_bounds__(32 * kBkWarps, 6) k_render_bwd_bucket(gs_config cfg, Ws ws, BwdArgs a, BucketWs bw) {
  // pair u = x + 16 r (x = column, r = row pair): pixels x + 32 r and x + 32 r + 16
  __shared__ float4 s_p0[128];                       // dL/dC_r (both pixels), dL/dC_g (both)
  __shared__ float4 s_p1[128];                       // dL/dC_b, dL/dD
  __shared__ float4 s_p2[128];                       // dL/dO, a.Y
  __shared__ uint32_t s_nc[256];                     // by pixel
  __shared__ uint32_t s_list[kBkWarps][128];         // u | reach(top) << 8 | reach(bottom) << 16
  __shared__ float4 s_ck[kBkWarps][32];              // (T top, T bottom, A top, A bottom) of 32 streamed pairs
  __shared__ float s_pre[kBkWarps][2][10][32];       // checkpoints of the next 32 pairs (double-buffered)
  __shared__ uint32_t s_max;
  __shared__ float s_loss[kBkWarps];
  if (ws.counters[kStatus] != 0) return;
  constexpr int NT = 32 * kBkWarps;
  const int64_t tile = blockIdx.x;
  const int v = (int)(tile / ws.tiles_per_view);
  const int t = (int)(tile - (int64_t)v * ws.tiles_per_view);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx0 = (t % ws.tiles_x) * kTile, ty0 = (t / ws.tiles_x) * kTile;
  const uint32_t start = ws.tile_start[tile], cnt = ws.tile_count[tile];
  const int64_t HW = (int64_t)ws.width * ws.height;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();

  // ---- pixel adjoints
  uint32_t mx = 0;
  float loss = 0.f;
  float* p0f = reinterpret_cast<float*>(s_p0);
  float* p1f = reinterpret_cast<float*>(s_p1);
  float* p2f = reinterpret_cast<float*>(s_p2);
  for (int lp = threadIdx.x; lp < 256; lp += NT) {
    const int x = tx0 + (lp & 15), y = ty0 + (lp >> 4);
    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float ay = 0.f;
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
    const int u = (lp & 15) + 16 * (lp >> 5), h = (lp >> 4) & 1;
    p0f[4 * u + h] = g[0];
    p0f[4 * u + 2 + h] = g[1];
    p1f[4 * u + h] = g[2];
    p1f[4 * u + 2 + h] = g[3];
    p2f[4 * u + h] = g[4];
    p2f[4 * u + 2 + h] = ay;
    s_nc[lp] = nc;
    mx = max(mx, nc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    loss += __shfl_xor_sync(kFull, loss, o);
  }
  if (lane == 0) {
    atomicMax(&s_max, mx);
    s_loss[warp] = loss;
  }
  __syncthreads();
  if (FUSED && a.loss && threadIdx.x == 0) {
    float tot = 0.f;
    for (int i = 0; i < kBkWarps; ++i) tot += s_loss[i];
    if (tot != 0.f) atomicAdd(a.loss + v, tot);
  }
  const uint32_t maxnc = min(s_max, cnt);
  const int nbk = (int)((maxnc + 31u) >> 5);
  const float4* rec = ws.records + 3 * (int64_t)v * ws.n;
  float4* adj = ws.adjoints + 3 * (int64_t)v * ws.n;
  const float a_max = cfg.alpha_max;
  const float lt = __log2f(cfg.alpha_min);
  const float ox = (float)tx0 + 0.5f, oy = (float)ty0 + 0.5f;
  uint32_t* list = s_list[warp];
  float4* ring = s_ck[warp];

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
    // a lane whose Gaussian lies past the list reaches no pixel
    const uint32_t lane_g = g_ok ? (uint32_t)lane : 64u;
    // the pixel pairs with a pixel whose contributors reach into this bucket, in order
    __syncwarp();
    uint32_t m = 0;
    const uint32_t kb = 32u * (uint32_t)k;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      const int u = 32 * c4 + lane;
      const int pt = (u & 15) + 32 * (u >> 4);
      const uint32_t n0 = s_nc[pt], n1 = s_nc[pt + 16];
      const uint32_t r0 = n0 > kb ? min(n0 - kb, 32u) : 0u, r1 = n1 > kb ? min(n1 - kb, 32u) : 0u;
      const bool in = (r0 | r1) != 0u;
      const unsigned b = __ballot_sync(kFull, in);
      if (in) list[m + __popc(b & ((1u << lane) - 1u))] = (uint32_t)u | (r0 << 8) | (r1 << 16);
      m += (uint32_t)__popc(b);
    }
    __syncwarp();
    const float* ck = bw.ckpt + ((int64_t)(start >> 5) + tile + k) * (5 * 256);
    // checkpoints of the streamed pairs, copied asynchronously into shared
    // memory one chunk of 32 pairs ahead (lane l copies pair l of the chunk)
    auto fetch = [&](uint32_t pq, int buf) {
      if (pq < m) {
        const uint32_t u = list[pq] & 255u;
        const uint32_t pt = (u & 15u) + 32u * (u >> 4);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          cp_async4(&s_pre[warp][buf][q][lane], ck + q * 256 + pt);
          cp_async4(&s_pre[warp][buf][5 + q][lane], ck + q * 256 + pt + 16);
        }
      }
      cp_async_commit();
    };
    fetch((uint32_t)lane, 0);
    const float2 cr = f2(c.x), cg = f2(c.y), cb = f2(c.z), dep = f2(g1.z), hc = f2(g1.x);
    // sums over the pixels: dp dx, dp dy, dp dx^2, dp dx dy, dp dy^2, dp (dp = dL/dpower,
    // zero where alpha is clamped), and dL/dD w, dL/dC w (w = alpha T); both pixels of a
    // pair share dx, so the dx moments take the pair sums
    float2 Q1 = f2(0.f), Q4 = Q1, Q5 = Q1, Qx = Q1, V6 = Q1, V7 = Q1, V8 = Q1, V9 = Q1;
    float q0 = 0.f, q2 = 0.f;
    float2 Tst = f2(0.f), Ast = f2(0.f);
    const uint32_t steps = m + 31u;
    // steps in unrolled groups of eight: a chunk of 32 starts only at the first of a group
    for (uint32_t s0 = 0; s0 < steps; s0 += 8) {
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
      const uint32_t s = s0 + u;
      if (s >= steps) break;
      if (u == 0 && (s & 31u) == 0) {
        const int buf = (int)((s >> 5) & 1u);
        cp_async_wait_all();  // this lane's copies of the chunk (issued 32 steps ago)
        __syncwarp();
        const uint32_t pq = s + (uint32_t)lane;
        if (pq < m) {
          const uint32_t u = list[pq] & 255u;
          const float4 a0 = s_p0[u], a1 = s_p1[u], a2 = s_p2[u];
          const float(*pr)[32] = s_pre[warp][buf];
          const float t0 = pr[0][lane], t1 = pr[5][lane];
          ring[lane] = make_float4(t0, t1,
                                   a0.x * pr[1][lane] + a0.z * pr[2][lane] + a1.x * pr[3][lane] +
                                       a1.z * pr[4][lane] + a2.x * (1.f - t0),
                                   a0.y * pr[6][lane] + a0.w * pr[7][lane] + a1.y * pr[8][lane] +
                                       a1.w * pr[9][lane] + a2.y * (1.f - t1));
        }
        __syncwarp();
        fetch(s + 32u + (uint32_t)lane, buf ^ 1);
      }
      const float tin0 = __shfl_up_sync(kFull, Tst.x, 1), tin1 = __shfl_up_sync(kFull, Tst.y, 1);
      const float ain0 = __shfl_up_sync(kFull, Ast.x, 1), ain1 = __shfl_up_sync(kFull, Ast.y, 1);
      const int q = (int)s - lane;
      if (q >= 0 && q < (int)m) {
        float2 T = make_float2(tin0, tin1), A = make_float2(ain0, ain1);
        if (lane == 0) {
          const float4 r4 = ring[q & 31];
          T = make_float2(r4.x, r4.y);
          A = make_float2(r4.z, r4.w);
        }
        const uint32_t e = list[q];
        const uint32_t u = e & 255u;
        const float px = ox + (float)(u & 15u);
        const float py = oy + (float)(2u * (u >> 4));
        // the exponent of the forward, operation for operation (col_terms, col_p2x2)
        const ColTerms ct = col_terms(g0, g1, px);
        const float2 p2 = col_p2x2(ct, make_float2(py, py + 1.f));
        const bool act0 = lane_g < ((e >> 8) & 255u) && p2.x >= lt, act1 = lane_g < (e >> 16) && p2.y >= lt;
        if (act0 | act1) {
          const float e0 = ex2_approx(p2.x), e1 = ex2_approx(p2.y);
          const float2 al = make_float2(act0 ? fminf(a_max, e0) : 0.f, act1 ? fminf(a_max, e1) : 0.f);
          // alpha = o exp(power): dL/dpower = dL/dalpha alpha, zero where alpha is clamped
          const float2 ag = make_float2(e0 > a_max ? 0.f : al.x, e1 > a_max ? 0.f : al.y);
          const float4 a0 = s_p0[u], a1 = s_p1[u], a2 = s_p2[u];
          const float2 ar = make_float2(a0.x, a0.y), agr = make_float2(a0.z, a0.w), ab = make_float2(a1.x, a1.y),
                       ad = make_float2(a1.z, a1.w);
          const float2 wg = fma2(ar, cr, fma2(agr, cg, fma2(ab, cb, fma2(ad, dep, make_float2(a2.x, a2.y)))));
          const float2 aT = mul2(al, T);
          A = fma2(aT, wg, A);
          const float2 om = fma2(al, f2(-1.f), f2(1.f));
          const float2 behind = fma2(A, f2(-1.f), make_float2(a2.z, a2.w));  // a.Y - A
          const float2 dA = fma2(mul2(behind, make_float2(rcp_approx(om.x), rcp_approx(om.y))), f2(-1.f),
                                 mul2(T, wg));
          T = mul2(T, om);
          const float2 dp = mul2(dA, ag);
          const float2 dy = make_float2(py - g0.y, py + 1.f - g0.y);
          const float2 dpy = mul2(dp, dy);
          const float dx = px - g0.x;
          Q5 = add2(Q5, dp);                 // sum dp
          Q1 = add2(Q1, dpy);                // sum dp dy
          Q4 = fma2(dpy, dy, Q4);            // sum dp dy^2
          Qx = fma2(dpy, f2(dx), Qx);        // sum dp dx dy
          const float dps = dp.x + dp.y;
          q0 = fmaf(dps, dx, q0);            // sum dp dx
          q2 = fmaf(dps * dx, dx, q2);       // sum dp dx^2
          V6 = fma2(ad, aT, V6);
          V7 = fma2(ar, aT, V7);
          V8 = fma2(agr, aT, V8);
          V9 = fma2(ab, aT, V9);
        }
        Tst = T;
        Ast = A;
      }
    }
    }
    if (g_ok) {
      // the same 2D adjoints as the pixel-parallel kernel's flush
      const float q1 = Q1.x + Q1.y, q3 = Qx.x + Qx.y, q4 = Q4.x + Q4.y, q5 = Q5.x + Q5.y, v6 = V6.x + V6.y,
                  v7 = V7.x + V7.y, v8 = V8.x + V8.y, v9 = V9.x + V9.y;
      const float gmx = -kLn2 * (2.f * g0.z * q0 + g0.w * q1);
      const float gmy = -kLn2 * (g0.w * q0 + 2.f * g1.x * q1);
      const float ga = -0.5f * q2, gb = -q3, gc = -0.5f * q4, go = q5 * g1.w;
      float4* dst = adj + 3 * (int64_t)gid;
      if (q0 != 0.f || q1 != 0.f || q2 != 0.f || q3 != 0.f) red_add4(dst, make_float4(gmx, gmy, ga, gb));
      if (q4 != 0.f || q5 != 0.f || v6 != 0.f) red_add4(dst + 1, make_float4(gc, go, v6, 0.f));
      if (v7 != 0.f || v8 != 0.f || v9 != 0.f) red_add4(dst + 2, make_float4(v7, v8, v9, 0.f));
    }
  }
}

cudaError_t launch_render_bwd_bucket(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                     const BwdArgs& a, const BucketWs& bw, cudaStream_t st) {
  cudaError_t err = launch_bwd_prologue(ws, a, st);
  if (err != cudaSuccess) return err;
  const unsigned ntiles = (unsigned)((int64_t)ws.views * ws.tiles_per_view);
  trace_begin(kKRenderBwdBucket, st);
  if (a.tgt_rgb) k_render_bwd_bucket<true><<<ntiles, 32 * kBkWarps, 0, st>>>(cfg, ws, a, bw);
  else k_render_bwd_bucket<false><<<ntiles, 32 * kBkWarps, 0, st>>>(cfg, ws, a, bw);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_preprocess_bwd(map, cams, cfg, ws, a, st);
}

}  // namespace gsb
