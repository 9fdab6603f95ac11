// Keyframe unpacking for the mapping step (Sec. "Additional Strategies" (e):
// keyframes move host -> device with asynchronous copies).  Camera images
// arrive as 8-bit RGB and the LiDAR depth map as its valid pixels only (a
// few percent of the image); this kernel expands them on the device into the
// FP32 planes the rasterizer's loss reads: colour c / 255, depth 0 where no
// LiDAR point projects.
#include "gs_internal.h"

namespace gsb {

// c / 255 (correctly rounded) for every byte value c, from a table each CTA
// fills once.  VEC: 16 bytes per thread and step (both pointers 16-byte
// aligned), the remaining n % 16 bytes one per thread.
template <bool VEC>
__global__ void __launch_bounds__(256) k_unpack_rgb(const uint8_t* __restrict__ rgb8, int64_t n,
                                                    float* __restrict__ rgb) {
  __shared__ float s_lut[256];
  s_lut[threadIdx.x] = __fdiv_rn((float)threadIdx.x, 255.f);
  __syncthreads();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nv = VEC ? n / 16 : 0;
  if (VEC) {
    const uint4* src = reinterpret_cast<const uint4*>(rgb8);
    float4* dst = reinterpret_cast<float4*>(rgb);
    for (int64_t i = tid; i < nv; i += stride) {
      const uint4 q = src[i];
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)  // bytes in address order: the low byte of each word first
        dst[4 * i + k] = make_float4(s_lut[w[k] & 255u], s_lut[(w[k] >> 8) & 255u], s_lut[(w[k] >> 16) & 255u],
                                     s_lut[w[k] >> 24]);
    }
  }
  for (int64_t i = 16 * nv + tid; i < n; i += stride) rgb[i] = s_lut[rgb8[i]];
}

__global__ void k_unpack_depth(const int32_t* __restrict__ idx, const float* __restrict__ val,
                               const int32_t* __restrict__ offsets, int V, int64_t hw, float* __restrict__ depth) {
  const int v = blockIdx.y;
  const int32_t b = offsets[v], e = offsets[v + 1];
  for (int32_t i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
    const int32_t p = idx[i];
    if (p >= 0 && p < hw) depth[v * hw + p] = val[i];
  }
}

cudaError_t launch_unpack_keyframes(const uint8_t* rgb8, int V, int H, int W, float* rgb, const int32_t* idx,
                                    const float* val, const int32_t* offsets, float* depth, cudaStream_t st) {
  const int64_t hw = (int64_t)H * W;
  const int64_t n = (int64_t)V * 3 * hw;
  const unsigned grid = (unsigned)sm_count() * 8;
  if (rgb8) {  // colour planes (none when the loss reads the 8-bit images itself)
    if (reinterpret_cast<uintptr_t>(rgb8) % 16 == 0 && reinterpret_cast<uintptr_t>(rgb) % 16 == 0)
      k_unpack_rgb<true><<<grid, 256, 0, st>>>(rgb8, n, rgb);
    else
      k_unpack_rgb<false><<<grid, 256, 0, st>>>(rgb8, n, rgb);
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || !depth) return err;
  if ((err = cudaMemsetAsync(depth, 0, (size_t)V * hw * sizeof(float), st)) != cudaSuccess) return err;
  if (!idx) return cudaSuccess;
  // about one point per thread for the few percent of pixels a LiDAR sweep hits
  const unsigned gx = (unsigned)((hw / 16 + 255) / 256);
  k_unpack_depth<<<dim3(gx < 1 ? 1u : gx, (unsigned)V), 256, 0, st>>>(idx, val, offsets, V, hw, depth);
  return cudaGetLastError();
}

}  // namespace gsb
