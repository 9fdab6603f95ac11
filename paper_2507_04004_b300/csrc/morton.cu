// Spatial storage order of the Gaussian map.
//
// The map's parameters are structure-of-arrays indexed by Gaussian.  A view
// sees a few tens of percent of the Gaussians, and when those are scattered
// through the arrays in random order nearly every 32-byte sector of every
// parameter row is fetched by the projection, the projection backward and
// the sparse Adam step (Sec. "Additional Strategies" (a): only the rendered
// Gaussians are updated).  Ordering the Gaussians along a space-filling curve
// of their means makes the Gaussians a view sees, and those of a tile,
// contiguous runs of the arrays.
//   gs_morton_order: the permutation sorting the Gaussians by the 30-bit
//     Morton code of their means (10 bits per axis over the map's bounding
//     box), ties by index (a stable radix sort);
//   gs_permute_rows: dst[r][i] = src[r][perm[i]] for SoA rows of 2- or 4-byte
//     elements, to apply it to the parameters and optimiser moments.
#include "gs_internal.h"
#include "radix.cuh"

namespace gsb {

// Scratch header words (uint32): [0] error word, [1] n, [2..7] tile tickets,
// [8..10] minimum of each axis and [11..13] maximum (order-preserving
// integers of the floats).
constexpr int kMortonHeader = 64;  // words, so the digit counts start 256-byte aligned


static size_t align256m(size_t x) { return (x + 255) & ~size_t(255); }

static size_t morton_layout(int64_t n, size_t* off_counts, size_t* off_tiles, size_t* off_k0, size_t* off_v0,
                            size_t* off_k1, size_t* off_v1, int64_t* tiles_max) {
  const int64_t tiles = (n + kRadixTileEntries - 1) / kRadixTileEntries;
  size_t off = align256m(kMortonHeader * sizeof(uint32_t));
  *off_counts = off;
  off += align256m(6 * 256 * sizeof(uint32_t));
  *off_tiles = off;
  off += align256m((size_t)4 * tiles * 256 * sizeof(uint32_t));
  *off_k0 = off;
  off += align256m((size_t)n * sizeof(uint32_t));
  *off_v0 = off;
  off += align256m((size_t)n * sizeof(uint32_t));
  *off_k1 = off;
  off += align256m((size_t)n * sizeof(uint32_t));
  *off_v1 = off;
  off += align256m((size_t)n * sizeof(uint32_t));
  *tiles_max = tiles;
  return off;
}

// Order-preserving map of floats to unsigned integers (and back).
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// The low 10 bits of x moved to bits 0, 3, 6, ..., 27.
__device__ __forceinline__ uint32_t spread_bits3(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void k_morton_reset(uint32_t* head, uint32_t* counts, uint32_t n) {
  for (int i = threadIdx.x; i < kMortonHeader; i += blockDim.x)
    head[i] = (i >= 8 && i < 11) ? 0xffffffffu : (i == 1 ? n : 0u);
  for (int i = threadIdx.x; i < 6 * 256; i += blockDim.x) counts[i] = 0;
}

// Bounding box of the finite means.
__global__ void __launch_bounds__(256) k_morton_bbox(const float* __restrict__ mean, int64_t n, uint32_t* head) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float m = mean[a * n + i];
      if (!isfinite(m)) continue;
      const uint32_t o = float_to_ordered(m);
      lo[a] = min(lo[a], o);
      hi[a] = max(hi[a], o);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(kFull, lo[a], o));
      hi[a] = max(hi[a], __shfl_xor_sync(kFull, hi[a], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(head + 8 + a, lo[a]);
      atomicMax(head + 11 + a, hi[a]);
    }
  }
}

// Morton code of every mean: per axis q = floor((m - lo) 1024 / (hi - lo))
// clamped to [0, 1023] (0 for a flat axis or a non-finite mean), the bits
// of x, y, z interleaved with x the most significant.
__global__ void __launch_bounds__(256) k_morton_codes(const float* __restrict__ mean, int64_t n,
                                                      const uint32_t* __restrict__ head, uint32_t* __restrict__ code,
                                                      uint32_t* __restrict__ idx) {
  float lo[3], scale[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = ordered_to_float(head[8 + a]);
    const float ext = __fsub_rn(ordered_to_float(head[11 + a]), lo[a]);
    scale[a] = ext > 0.f ? __fdiv_rn(1024.f, ext) : 0.f;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float m = mean[a * n + i];
      const float t = isfinite(m) ? floorf(__fmul_rn(__fsub_rn(m, lo[a]), scale[a])) : 0.f;
      q[a] = (uint32_t)fminf(fmaxf(t, 0.f), 1023.f);
    }
    code[i] = (spread_bits3(q[0]) << 2) | (spread_bits3(q[1]) << 1) | spread_bits3(q[2]);
    idx[i] = (uint32_t)i;
  }
}

struct CodeDigit {
  __device__ __forceinline__ uint32_t operator()(uint32_t key, uint32_t, int pass) const {
    return (key >> (8 * pass)) & 255u;
  }
};

__global__ void __launch_bounds__(256) k_permute_rows(const unsigned char* __restrict__ src,
                                                      unsigned char* __restrict__ dst, int64_t rows, int64_t n,
                                                      int elem_bytes, const uint32_t* __restrict__ perm) {
  const int64_t total = rows * n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / n, i = k - r * n;
    const uint32_t pi = perm[i];
    if (pi >= (uint64_t)n) continue;  // not a permutation of [0, n): the slot is left as it is
    const int64_t from = r * n + pi;
    if (elem_bytes == 4)
      reinterpret_cast<uint32_t*>(dst)[k] = reinterpret_cast<const uint32_t*>(src)[from];
    else
      reinterpret_cast<uint16_t*>(dst)[k] = reinterpret_cast<const uint16_t*>(src)[from];
  }
}

}  // namespace gsb

using namespace gsb;

extern "C" size_t gs_morton_scratch_bytes(int64_t n) {
  if (n < 1 || n >= (int64_t(1) << 30)) return 0;
  size_t a, b, c, d, e, f;
  int64_t t;
  return morton_layout(n, &a, &b, &c, &d, &e, &f, &t);
}

extern "C" gs_status gs_morton_order(const float* mean_dev, int64_t n, void* scratch, uint32_t* perm_out,
                                     gs_stream_t stream) {
  if (!mean_dev || !scratch || !perm_out || n < 1) return GS_ERR_ARG;
  if (n >= (int64_t(1) << 30)) return GS_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(scratch) & 255u) != 0) return GS_ERR_ARG;
  size_t oc, ot, ok0, ov0, ok1, ov1;
  int64_t tiles;
  morton_layout(n, &oc, &ot, &ok0, &ov0, &ok1, &ov1, &tiles);
  char* b = static_cast<char*>(scratch);
  uint32_t* head = reinterpret_cast<uint32_t*>(b);
  uint32_t* k0 = reinterpret_cast<uint32_t*>(b + ok0);
  uint32_t* v0 = reinterpret_cast<uint32_t*>(b + ov0);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(b + ok1);
  uint32_t* v1 = reinterpret_cast<uint32_t*>(b + ov1);
  RadixScratch rs;
  rs.n = head + 1;
  rs.status = head;
  rs.counts = reinterpret_cast<uint32_t*>(b + oc);
  rs.tiles = reinterpret_cast<uint32_t*>(b + ot);
  rs.tickets = head + 2;
  rs.tiles_max = tiles;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)sm_count() * 4;
  k_morton_reset<<<1, 256, 0, st>>>(head, rs.counts, (uint32_t)n);
  k_morton_bbox<<<grid, 256, 0, st>>>(mean_dev, n, head);
  k_morton_codes<<<grid, 256, 0, st>>>(mean_dev, n, head, k0, v0);
  k_radix_counts<<<grid, kRadixThreads, 0, st>>>(rs, CodeDigit{}, 4, k0, v0);
  // passes 0 and 2 go to (k1, v1), 1 to (k0, v0), the last one straight into perm_out
  k_radix_pass<<<grid, kRadixThreads, 0, st>>>(rs, CodeDigit{}, 0, k0, v0, k1, v1);
  k_radix_pass<<<grid, kRadixThreads, 0, st>>>(rs, CodeDigit{}, 1, k1, v1, k0, v0);
  k_radix_pass<<<grid, kRadixThreads, 0, st>>>(rs, CodeDigit{}, 2, k0, v0, k1, v1);
  k_radix_pass<<<grid, kRadixThreads, 0, st>>>(rs, CodeDigit{}, 3, k1, v1, k0, perm_out);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status gs_permute_rows(const void* src_dev, void* dst_dev, int64_t rows, int64_t n, int32_t elem_bytes,
                                     const uint32_t* perm_dev, gs_stream_t stream) {
  if (!src_dev || !dst_dev || !perm_dev || rows < 0 || n < 1 || (elem_bytes != 2 && elem_bytes != 4))
    return GS_ERR_ARG;
  if (src_dev == dst_dev) return GS_ERR_ARG;
  if (rows == 0) return GS_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_permute_rows<<<(unsigned)sm_count() * 8, 256, 0, st>>>(static_cast<const unsigned char*>(src_dev),
                                                           static_cast<unsigned char*>(dst_dev), rows, n, elem_bytes,
                                                           perm_dev);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
