// Map expansion (Sec. "Expansion of Gaussian Map"): the opacity map O of a
// new keyframe is rendered (Eq. rendered_opacity), the mask O < tau marks
// the newly observed image regions, and only the keyframe's 3D points that
// project into those regions initialise new Gaussians.
//
// Selection keeps the input order of the points (flags, one exclusive scan,
// scatter), so the new Gaussians come out in a deterministic order.
// Initialisation (the paper takes it from its predecessors; the values are
// readings): mean = the point, isotropic scale of two pixels at the point's
// depth, identity rotation, opacity init_opacity, SH DC from the point's
// colour (colour = 0.5 + Y_00 DC), higher SH zero.
#include <cmath>

#include "gs_internal.h"

namespace gsb {

__device__ __forceinline__ bool point_pixel(const gs_camera& c, float x, float y, float z, int W, int H, float near,
                                            int* px, int* py, float* depth) {
  const float qx = __fmaf_rn(c.R[0], x, __fmaf_rn(c.R[1], y, __fmaf_rn(c.R[2], z, c.t[0])));
  const float qy = __fmaf_rn(c.R[3], x, __fmaf_rn(c.R[4], y, __fmaf_rn(c.R[5], z, c.t[1])));
  const float qz = __fmaf_rn(c.R[6], x, __fmaf_rn(c.R[7], y, __fmaf_rn(c.R[8], z, c.t[2])));
  if (!(qz > near)) return false;
  const float u = c.fx * qx / qz + c.cx, v = c.fy * qy / qz + c.cy;
  const float fu = floorf(u), fv = floorf(v);
  if (!(fu >= 0.f && fu < (float)W && fv >= 0.f && fv < (float)H)) return false;
  *px = (int)fu;
  *py = (int)fv;
  *depth = qz;
  return true;
}

__global__ void k_expand_flags(const float* __restrict__ pts, int64_t P, const gs_camera* __restrict__ cam,
                               const float* __restrict__ opac, int H, int W, float tau, float near,
                               uint32_t* __restrict__ flags) {
  const gs_camera c = *cam;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    int px, py;
    float d;
    const bool in = point_pixel(c, pts[i], pts[P + i], pts[2 * P + i], W, H, near, &px, &py, &d);
    flags[i] = (in && opac[(int64_t)py * W + px] < tau) ? 1u : 0u;
  }
}

// Exclusive scan of the flags by one CTA (warp-owned segments, coalesced).
__global__ void __launch_bounds__(1024) k_expand_scan(const uint32_t* __restrict__ flags, int64_t P,
                                                      uint32_t* __restrict__ offs, uint32_t* __restrict__ count) {
  constexpr int NW = 32;
  __shared__ uint32_t wbase[NW + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (P + NW - 1) / NW;
  const int64_t b = min(P, (int64_t)warp * seg), e = min(P, b + seg);
  uint32_t s = 0;
  for (int64_t i = b + lane; i < e; i += 32) s += flags[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if (lane == 0) wbase[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = wbase[lane];
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    wbase[lane] = inc - v;
    if (lane == 31) wbase[NW] = inc;
  }
  __syncthreads();
  uint32_t run = wbase[warp];
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane;
    const uint32_t f = i < e ? flags[i] : 0u;
    uint32_t inc = f;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (i < e) offs[i] = run + inc - f;
    run += __shfl_sync(kFull, inc, 31);
  }
  if (threadIdx.x == 0) *count = wbase[NW];
}

__global__ void k_expand_scatter(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ offs, int64_t P,
                                 int32_t* __restrict__ out_idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) out_idx[offs[i]] = (int32_t)i;
}

// New Gaussians from selected points: n_new = *count (device), written at
// offset `first` of the destination map arrays (capacity checked by the host).
__global__ void k_expand_init(const float* __restrict__ pts, const float* __restrict__ rgb, int64_t P,
                              const int32_t* __restrict__ idx, const uint32_t* __restrict__ count,
                              const gs_camera* __restrict__ cam, int64_t first, int64_t n_dst, int32_t K,
                              float logit_init, gs_param_set dst) {
  const gs_camera c = *cam;
  const uint32_t nn = *count;
  constexpr float kY00 = 0.28209479177387814f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[j];
    const int64_t g = first + j;
    if (g >= n_dst) break;
    const float x = pts[i], y = pts[P + i], z = pts[2 * P + i];
    const float qz = __fmaf_rn(c.R[6], x, __fmaf_rn(c.R[7], y, __fmaf_rn(c.R[8], z, c.t[2])));
    const float s = logf(2.f * qz / c.fx);  // two pixels across at the point's depth
    dst.mean[g] = x;
    dst.mean[n_dst + g] = y;
    dst.mean[2 * n_dst + g] = z;
    for (int k = 0; k < 3; ++k) dst.log_scale[k * n_dst + g] = s;
    dst.quat[g] = 1.f;
    dst.quat[n_dst + g] = 0.f;
    dst.quat[2 * n_dst + g] = 0.f;
    dst.quat[3 * n_dst + g] = 0.f;
    dst.logit_opacity[g] = logit_init;
    for (int ch = 0; ch < 3; ++ch) dst.sh_dc[ch * n_dst + g] = (rgb[ch * P + i] - 0.5f) / kY00;
    if (dst.sh_rest)
      for (int r = 0; r < 3 * (K - 1); ++r) dst.sh_rest[(int64_t)r * n_dst + g] = 0.f;
  }
}

size_t expand_scratch_bytes(int64_t P) {
  return 2 * (((size_t)P * sizeof(uint32_t) + 255) / 256 * 256) + 256;
}

cudaError_t launch_expand_select(const float* pts, int64_t P, const gs_camera* cam, const float* opac, int H, int W,
                                 float tau, float near, void* scratch, int32_t* out_idx, uint32_t* count,
                                 cudaStream_t st) {
  uint32_t* flags = static_cast<uint32_t*>(scratch);
  uint32_t* offs = flags + ((size_t)P * sizeof(uint32_t) + 255) / 256 * 64;
  const int64_t need = (P + 255) / 256;
  const unsigned grid = (unsigned)(need < sm_count() * 8 ? need : sm_count() * 8);
  k_expand_flags<<<grid, 256, 0, st>>>(pts, P, cam, opac, H, W, tau, near, flags);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_expand_scan<<<1, 1024, 0, st>>>(flags, P, offs, count);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_expand_scatter<<<grid, 256, 0, st>>>(flags, offs, P, out_idx);
  return cudaGetLastError();
}

cudaError_t launch_expand_init(const float* pts, const float* rgb, int64_t P, const int32_t* idx,
                               const uint32_t* count, const gs_camera* cam, int64_t first, int64_t n_dst,
                               int32_t sh_degree, float logit_init, const gs_param_set& dst, cudaStream_t st) {
  const int64_t need = (P + 255) / 256;
  const unsigned grid = (unsigned)(need < sm_count() * 8 ? (need > 0 ? need : 1) : sm_count() * 8);
  k_expand_init<<<grid, 256, 0, st>>>(pts, rgb, P, idx, count, cam, first, n_dst,
                                      (sh_degree + 1) * (sh_degree + 1), logit_init, dst);
  return cudaGetLastError();
}

}  // namespace gsb
