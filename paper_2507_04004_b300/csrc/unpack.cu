// Keyframe unpacking for the mapping step (Sec. "Additional Strategies" (e):
// keyframes move host -> device with asynchronous copies).  Camera images
// arrive as 8-bit RGB and the LiDAR depth map as its valid pixels only (a
// few percent of the image); this kernel expands them on the device into the
// FP32 planes the rasterizer's loss reads: colour c / 255, depth 0 where no
// LiDAR point projects.
#include "gs_internal.h"

namespace gsb {

__global__ void k_unpack_rgb(const uint8_t* __restrict__ rgb8, int64_t n, float* __restrict__ rgb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rgb[i] = __fdiv_rn((float)rgb8[i], 255.f);
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
  k_unpack_rgb<<<grid, 256, 0, st>>>(rgb8, n, rgb);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || !depth) return err;
  if ((err = cudaMemsetAsync(depth, 0, (size_t)V * hw * sizeof(float), st)) != cudaSuccess) return err;
  if (!idx) return cudaSuccess;
  k_unpack_depth<<<dim3(16, (unsigned)V), 256, 0, st>>>(idx, val, offsets, V, hw, depth);
  return cudaGetLastError();
}

}  // namespace gsb
