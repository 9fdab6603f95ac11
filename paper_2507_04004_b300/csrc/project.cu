// Projection and SH colour of every (view, Gaussian), with the tile box and
// the row-item counts that the binning (binning.cu) starts from.
//
// arxiv 2507.04004, Sec. "3D Gaussian Splatting Representation":
//   mu_hat = R mu + t, d = e3^T mu_hat, mu' = pi_c(mu_hat / d),
//   Sigma' = J R Sigma R^T J^T (+ dilation), Sigma = R_g S S^T R_g^T,
//   colour from SH at the direction camera centre -> mean;
// Sec. "Fast Tile-based Culling": keep a tile iff the highest alpha the
// Gaussian reaches at one of its pixels is >= 1/255.  Sec. "Additional
// Strategies" (d): lanes carry a validity flag to one common exit and whole
// warps whose Gaussians are all cut skip the rest.
//
// The projection also writes, per view, the number of row items (one per
// (Gaussian, tile row of its box)) of every tile row as differences, and the
// compact list of visible entries with their depth keys; binning.cu takes it
// from there.
#include "gs_internal.h"

namespace gsb {

constexpr int kMaxBuckets = 4096;  // buckets counted in shared memory (else global atomics)
constexpr int kCamChunk = 32;      // views whose cameras k_project holds in shared memory at a time
constexpr int kCamF4 = 7;          // float4 per staged camera

// A view's camera as k_project reads it, with the per-view constants of its
// tests precomputed once per CTA instead of once per (Gaussian, view):
//   [0..2] rows of R with t, [3] fx fy cx cy, [4] the clamp limits of x/z and
//   y/z and |fx| |r0|, |fx| |r2|, [5] |fy| |r1|, |fy| |r2|, [6] the centre -R^T t.
__device__ __forceinline__ void stage_cam(const gs_camera* cams, int v, const gs_config& cfg, int width, int height,
                                          float4* dst) {
  const Cam c = load_cam(cams, v);
  const float limx = cfg.fov_clamp * 0.5f * (float)width / c.fx;
  const float limy = cfg.fov_clamp * 0.5f * (float)height / c.fy;
  const float n0 = sqrtf(c.R[0] * c.R[0] + c.R[1] * c.R[1] + c.R[2] * c.R[2]);
  const float n1 = sqrtf(c.R[3] * c.R[3] + c.R[4] * c.R[4] + c.R[5] * c.R[5]);
  const float n2 = sqrtf(c.R[6] * c.R[6] + c.R[7] * c.R[7] + c.R[8] * c.R[8]);
  const float3 cw = camera_centre(c);
  dst[0] = make_float4(c.R[0], c.R[1], c.R[2], c.t[0]);
  dst[1] = make_float4(c.R[3], c.R[4], c.R[5], c.t[1]);
  dst[2] = make_float4(c.R[6], c.R[7], c.R[8], c.t[2]);
  dst[3] = make_float4(c.fx, c.fy, c.cx, c.cy);
  dst[4] = make_float4(limx, limy, fabsf(c.fx) * n0, fabsf(c.fx) * n2);
  dst[5] = make_float4(fabsf(c.fy) * n1, fabsf(c.fy) * n2, 0.f, 0.f);
  dst[6] = make_float4(cw.x, cw.y, cw.z, 0.f);
}

__device__ __forceinline__ Cam staged_cam(const float4* p) {
  Cam c;
  const float4 a = p[0], b = p[1], d = p[2], f = p[3];
  c.R[0] = a.x; c.R[1] = a.y; c.R[2] = a.z; c.t[0] = a.w;
  c.R[3] = b.x; c.R[4] = b.y; c.R[5] = b.z; c.t[1] = b.w;
  c.R[6] = d.x; c.R[7] = d.y; c.R[8] = d.z; c.t[2] = d.w;
  c.fx = f.x; c.fy = f.y; c.cx = f.z; c.cy = f.w;
  return c;
}

template <int DEG, bool BF16>
__global__ void __launch_bounds__(256, 3) k_project(gs_map map, const gs_camera* __restrict__ cams, gs_config cfg,
                                                 Ws ws) {
  __shared__ uint32_t s_bucket[kMaxBuckets];
  // FP32 SH: each thread's 3K coefficients are copied asynchronously into its
  // own shared-memory column when it starts a Gaussian, so the DRAM latency
  // overlaps the first view's projection (dynamic shared memory, 3K x 256 floats)
  extern __shared__ float4 s_dyn[];
  constexpr int K = (DEG + 1) * (DEG + 1);
  float* s_shc = reinterpret_cast<float*>(s_dyn);
  // cameras of the current chunk of views, after the SH columns; then each
  // warp's visible entries of its current batch and chunk (32 x chunk slots
  // per warp), written out under one global reservation per warp and chunk
  float4* s_cam = s_dyn + (BF16 ? 0 : 3 * K * 256 / 4);
  const int wcap = 32 * min(ws.views, kCamChunk);
  uint32_t* w_vis = reinterpret_cast<uint32_t*>(s_cam + kCamChunk * kCamF4) + (threadIdx.x >> 5) * wcap;
  const int64_t n = ws.n;
  const int nb = ws.views * ws.tiles_y;
  const bool smem_buckets = nb <= kMaxBuckets;
  if (smem_buckets)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_bucket[i] = 0;
  const bool one_chunk = ws.views <= kCamChunk;  // staged once; else per chunk between barriers
  if (one_chunk)
    for (int i = threadIdx.x; i < ws.views; i += blockDim.x)
      stage_cam(cams, i, cfg, ws.width, ws.height, s_cam + kCamF4 * i);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // One thread per Gaussian, all views in turn: the parameters are read and
  // activated once, and the SH rows it reads again for later views are still
  // in cache.  Whole warps step together so that warp votes see all 32 lanes.
  // CTAs take chunks of blockDim.x Gaussians by ticket: with the map in a
  // spatial order, a chunk is either mostly seen by some view or mostly not,
  // so a static split would leave SMs idle at the end.  Thread 0 takes the
  // next ticket when a chunk starts; the atomic's round trip overlaps it.
  __shared__ uint32_t s_chunk;
  uint32_t next_chunk = 0;
  if (threadIdx.x == 0) next_chunk = atomicAdd(ws.counters + kProjectTicket, 1u);
  for (;;) {
    if (threadIdx.x == 0) {
      s_chunk = next_chunk;
      next_chunk = atomicAdd(ws.counters + kProjectTicket, 1u);
    }
    __syncthreads();
    const int64_t base = (int64_t)s_chunk * blockDim.x;
    if (base >= n) break;  // the whole CTA
    const int64_t g = base + threadIdx.x;
    const bool in_range = g < n;
    float mw[3] = {0.f, 0.f, 1.f};
    float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f, ls[3] = {0.f, 0.f, 0.f}, logit = 0.f;
    if (in_range) {
      mw[0] = map.mean[g];
      mw[1] = map.mean[n + g];
      mw[2] = map.mean[2 * n + g];
      qw = map.quat[g]; qx = map.quat[n + g]; qy = map.quat[2 * n + g]; qz = map.quat[3 * n + g];
      ls[0] = map.log_scale[g]; ls[1] = map.log_scale[n + g]; ls[2] = map.log_scale[2 * n + g];
      logit = map.logit_opacity[g];
    }
    // FP32 SH: the copy into this thread's shared-memory column is issued once
    // the cheap candidate test below finds a view the Gaussian may reach, so
    // the coefficients of Gaussians no view sees are never read
    bool sh_pending = !BF16 && in_range;
    if (!BF16) cp_async_wait_all();  // the previous Gaussian's copies (long done) before the column is refilled
    const float qq = qw * qw + qx * qx + qy * qy + qz * qz;
    const bool g_ok = in_range && qq > 0.f;
    const float qi = g_ok ? rsqrtf(qq) : 1.f;
    float Rg[3][3];
    quat_to_rot(qw * qi, qx * qi, qy * qi, qz * qi, Rg);
    float sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = expf(ls[k]);
    const float o = 1.f / (1.f + expf(-logit));
    const float q_thr = 2.f * logf(o / cfg.alpha_min);
    bool seen = false;  // a non-empty box in some view
    // Views are taken 32 at a time.  A cheap pass marks each lane's candidate
    // views: in front of the near plane and not provably off-screen.  The
    // screen half-width of the box is sqrt(q_thr Sigma'_xx) with Sigma'_xx <=
    // s_max^2 |m0|^2 + dilation and |m0| <= |j00| |r0| + |j02| |r2| (r the
    // camera's rows); the bound below adds a relative and a one-pixel margin
    // for rounding, so it only drops views that the exact test drops.  The
    // full projection then runs over each lane's candidates only, so that
    // lanes are not left idle when a Gaussian is outside most views.
    const float s2max = fmaxf(sc[0], fmaxf(sc[1], sc[2])) * fmaxf(sc[0], fmaxf(sc[1], sc[2]));
    const float Wf = (float)(ws.width - 1), Hf = (float)(ws.height - 1);
    for (int v0 = 0; v0 < ws.views; v0 += kCamChunk) {
      const int nv = min(kCamChunk, ws.views - v0);
      if (!one_chunk) {
        __syncthreads();  // everyone is done with the previous chunk's cameras
        for (int i = threadIdx.x; i < nv; i += blockDim.x)
          stage_cam(cams, v0 + i, cfg, ws.width, ws.height, s_cam + kCamF4 * i);
        __syncthreads();
      }
      uint32_t cand = 0;
      int wn = 0;  // entries in this warp's list (warp-uniform)
      for (int j = 0; j < nv; ++j) {
        const int v = v0 + j;
        const float4* cp = s_cam + kCamF4 * j;
        const Cam cam = staged_cam(cp);
        const float3 mh = to_camera(cam, mw[0], mw[1], mw[2]);
        bool c = g_ok && q_thr > 0.f && mh.z > cfg.near_z;
        if (c) {
          const float iz = 1.f / mh.z;
          const float mx = __fmaf_rn(cam.fx * mh.x, iz, cam.cx);
          const float my = __fmaf_rn(cam.fy * mh.y, iz, cam.cy);
          const float4 k4 = cp[4], k5 = cp[5];
          const float txc = fminf(k4.x, fmaxf(-k4.x, mh.x * iz));
          const float tyc = fminf(k4.y, fmaxf(-k4.y, mh.y * iz));
          // |fx / z| |r0| + |fx x/z / z| |r2| (z > 0), and the same in y
          const float a0 = iz * (k4.z + fabsf(txc) * k4.w);
          const float a1 = iz * (k5.x + fabsf(tyc) * k5.y);
          const float hxb = 1.001f * sqrtf(q_thr * (1.001f * s2max * a0 * a0 + cfg.dilation)) + 1.f;
          const float hyb = 1.001f * sqrtf(q_thr * (1.001f * s2max * a1 * a1 + cfg.dilation)) + 1.f;
          if (mx - hxb - 1.5f > Wf + 1.f || mx + hxb + 0.5f < -1.f || my - hyb - 1.5f > Hf + 1.f ||
              my + hyb + 0.5f < -1.f)
            c = false;
        }
        if (c) cand |= 1u << j;
        else if (in_range) ws.rects[(int64_t)v * n + g] = empty_rect();
      }
      if (!BF16 && sh_pending && cand != 0) {
        sh_pending = false;
        const float* dc = static_cast<const float*>(map.sh_dc);
        const float* rest = static_cast<const float*>(map.sh_rest);
#pragma unroll
        for (int q = 0; q < 3 * K; ++q)
          cp_async4(s_shc + q * blockDim.x + threadIdx.x, q < 3 ? dc + q * n + g : rest + (int64_t)(q - 3) * n + g);
        cp_async_commit();
      }
      // warp-uniform loop (the list append below takes a ballot of all lanes)
      while (__any_sync(kFull, cand != 0)) {
        const bool act = cand != 0;
        const int v = act ? v0 + __ffs(cand) - 1 : v0;
        cand &= cand - 1;
        const int64_t e = (int64_t)v * n + g;
        const float4* cp = s_cam + kCamF4 * (v - v0);
        const Cam cam = staged_cam(cp);
        const float3 mh = to_camera(cam, mw[0], mw[1], mw[2]);
        bool ok = act && g_ok && (mh.z > cfg.near_z);
        const float z = ok ? mh.z : 1.f;
        const float iz = 1.f / z;
        const float mx = __fmaf_rn(cam.fx * mh.x, iz, cam.cx);
        const float my = __fmaf_rn(cam.fy * mh.y, iz, cam.cy);
        // affine Jacobian of the projection with x/z, y/z clamped
        const float4 k4 = cp[4];
        const float limx = k4.x, limy = k4.y;
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
        // U = S R_g^T m0, V = S R_g^T m1; Sigma' = [[U.U, U.V], [U.V, V.V]] + dil I
        float U[3], Vv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float s = sc[k];
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
        ok = ok && q_thr > 0.f && ca > 0.f && cc > 0.f;

        // Tile box from the axis-aligned extent of the ellipse q <= q_thr
        // (|dx| <= sqrt(q_thr Sigma'_xx), |dy| <= sqrt(q_thr Sigma'_yy)), one pixel of slack.
        int tx0 = 1, ty0 = 0, tx1 = 0, ty1 = 0;
        if (ok) {
          const float hx = sqrtf(q_thr * A), hy = sqrtf(q_thr * C);
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
          const float4 cw = cp[6];
          float dx = mw[0] - cw.x, dy = mw[1] - cw.y, dz = mw[2] - cw.z;
          const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
          dx *= inv; dy *= inv; dz *= inv;
          float Y[16];
          sh_basis<DEG>(dx, dy, dz, Y);
          if (!BF16) cp_async_wait_all();
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float cf = BF16 ? sh_coeff<BF16>(map.sh_dc, map.sh_rest, n, g, k, ch)
                                    : s_shc[(k == 0 ? ch : 3 * k + ch) * blockDim.x + threadIdx.x];
              acc += cf * Y[k];
            }
            rgb[ch] = fmaxf(acc, 0.f);
          }
        }

        // Single exit: record, cleared adjoint slot, tile box, row-item counts.
        if (ok) {
          float4* rec = ws.records + 3 * e;
          rec[0] = make_float4(mx, my, ca, cb);
          rec[1] = make_float4(cc, o, mh.z, q_thr);
          rec[2] = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
          float4* adj = ws.adjoints + 3 * e;
          adj[0] = adj[1] = adj[2] = make_float4(0.f, 0.f, 0.f, 0.f);
          // the entry's tile rows ty0..ty1 counted as a difference, +1 at ty0
          // and -1 after ty1 (the bucket scan sums them per view): two atomics
          // however many rows the box spans
          uint32_t* bc = (smem_buckets ? s_bucket : ws.bucket_count) + v * ws.tiles_y;
          atomicAdd(bc + ty0, 1u);
          if (ty1 + 1 < ws.tiles_y) atomicAdd(bc + ty1 + 1, 0xffffffffu);
        }
        if (act) ws.rects[e] = ok ? pack_rect(tx0, ty0, tx1, ty1) : empty_rect();
        // Append visible entries to the warp's list (positions by ballot).
        const unsigned vis = __ballot_sync(kFull, ok);
        if (ok) w_vis[wn + __popc(vis & ((1u << lane) - 1u))] = (uint32_t)e;
        wn += __popc(vis);
        seen |= ok;
      }
      // The warp's visible entries of this batch and chunk go to the compact
      // list under one global reservation (one hot counter otherwise takes an
      // atomic per warp step from every SM).
      if (wn) {
        uint32_t gb = 0;
        if (lane == 0) gb = atomicAdd(ws.counters + kVisibleCount, (uint32_t)wn);
        gb = __shfl_sync(kFull, gb, 0);
        __syncwarp();  // every lane's list entries before the reads below
        for (int i = lane; i < wn; i += 32) {
          const uint32_t e = w_vis[i];
          ws.visible[gb + i] = e;
          // the entry's depth key (its record was written by this warp before the __syncwarp)
          ws.vis_key[gb + i] = __float_as_uint(ws.records[3 * (int64_t)e + 1].z);
        }
        __syncwarp();  // read before the next chunk refills the list
      }
    }
    // Gaussians seen by some view, for the backward projection pass (one
    // atomic per warp; a warp's Gaussians stay consecutive in the list)
    const unsigned sn = __ballot_sync(kFull, seen);
    if (sn) {
      const int leader = __ffs(sn) - 1;
      uint32_t slot = 0;
      if (lane == leader) slot = atomicAdd(ws.counters + kGaussCount, (uint32_t)__popc(sn));
      slot = __shfl_sync(kFull, slot, leader);
      if (seen) ws.gauss_list[slot + __popc(sn & ((1u << lane) - 1u))] = (uint32_t)g;
    }
    __syncthreads();  // every thread has read s_chunk before thread 0 rewrites it
  }
  if (smem_buckets) {
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (s_bucket[i]) atomicAdd(ws.bucket_count + i, s_bucket[i]);
  }
}

template <int DEG, bool BF16>
static cudaError_t launch_project_t(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                    cudaStream_t st) {
  const int64_t need = (ws.n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 3;  // the CTAs resident at once (registers: 3 per SM)
  const unsigned grid = (unsigned)(need < cap ? need : cap);
  const size_t smem = (BF16 ? 0 : (size_t)3 * (DEG + 1) * (DEG + 1) * 256 * sizeof(float)) +
                      (size_t)kCamChunk * kCamF4 * sizeof(float4) +
                      (size_t)256 * (ws.views < kCamChunk ? ws.views : kCamChunk) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_project<DEG, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trace_begin(kKProject, st);
  k_project<DEG, BF16><<<grid, 256, smem, st>>>(map, cams, cfg, ws);
  trace_end(st);
  return cudaGetLastError();
}

cudaError_t launch_project(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                           cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(ws.counters, 0, 16 * sizeof(uint32_t), st);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(ws.tile_count, 0, (size_t)ws.views * ws.tiles_per_view * sizeof(uint32_t), st);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(ws.bucket_count, 0, (size_t)ws.views * ws.tiles_y * sizeof(uint32_t), st);
  if (err != cudaSuccess) return err;
  const bool bf = map.sh_bf16 != 0;
  switch (map.sh_degree) {
    case 0: return bf ? launch_project_t<0, true>(map, cams, cfg, ws, st) : launch_project_t<0, false>(map, cams, cfg, ws, st);
    case 1: return bf ? launch_project_t<1, true>(map, cams, cfg, ws, st) : launch_project_t<1, false>(map, cams, cfg, ws, st);
    case 2: return bf ? launch_project_t<2, true>(map, cams, cfg, ws, st) : launch_project_t<2, false>(map, cams, cfg, ws, st);
    default: return bf ? launch_project_t<3, true>(map, cams, cfg, ws, st) : launch_project_t<3, false>(map, cams, cfg, ws, st);
  }
}

}  // namespace gsb
