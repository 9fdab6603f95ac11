// D-SSIM term of the mapping loss (Sec. "Map Optimization") and of the
// tracking loss (Eq. tracking_loss, Sec. "Camera Factor (Option 2)"), which the
// paper takes from 3D Gaussian Splatting: per channel, SSIM of Wang et al.
// under an 11 x 11 Gaussian window (sigma 1.5, zero padding at the borders,
// C1 = 0.01^2, C2 = 0.03^2) and D = 1 - mean SSIM over a view.  Sec.
// "Additional Strategies" (c) computes it with separable Gaussian filters;
// so does this file: each 32 x 32 output tile stages its inputs with a 5-pixel
// halo in shared memory, filters rows then columns, and the backward pass
// filters the three per-pixel derivative maps the forward pass leaves behind.
#include <cmath>

#include "gs_internal.h"

namespace gsb {

namespace {

constexpr int kT = 32;             // output tile edge
constexpr int kR = 5;              // window radius
constexpr int kS = kT + 2 * kR;    // staged edge (42)
constexpr int kS2 = kS / 2;        // staged row pairs (21)
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Win {
  // normalised 1D Gaussian (the 2D window is its outer product), each weight
  // twice so that the packed FP32 pair instructions take it as it stands
  float2 w[2 * kR + 1];
};

// 4-byte asynchronous copy into shared memory, zero-filled when `in` is
// false (no global byte is read then; `src` must still be a valid address).
__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool in) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(in ? 4 : 0) : "memory");
}

// Stage one plane over the tile and its 5-pixel halo (zero outside the
// image) with rows paired, s[i][c] = (v[2i][c], v[2i + 1][c]), so that the
// row filter handles two rows per packed FP32x2 instruction.  The copies are
// asynchronous (all of a thread's loads in flight at once); the caller waits
// with cp_async_wait_all() and a barrier.
__device__ __forceinline__ void stage_pairs(const float* __restrict__ plane, int H, int W, int x0, int y0,
                                            float2 (*s)[kS]) {
  for (int i = threadIdx.x; i < kS2 * kS; i += blockDim.x) {
    const int rp = i / kS, c = i - rp * kS;
    const int gx = x0 + c, gy = y0 + 2 * rp;
    const bool cx = gx >= 0 && gx < W;
    const bool ia = cx && gy >= 0 && gy < H, ib = cx && gy + 1 >= 0 && gy + 1 < H;
    float* dst = reinterpret_cast<float*>(&s[rp][c]);
    cp_async4_zfill(dst, ia ? plane + (int64_t)gy * W + gx : plane, ia);
    cp_async4_zfill(dst + 1, ib ? plane + (int64_t)(gy + 1) * W + gx : plane, ib);
  }
}

// Row filter of NM maps formed from the staged planes by map_of (two rows and
// four output columns per thread: each of the 14 inputs is loaded and its
// products formed once), into out[m][row][col] for the kS rows and kT columns.
template <int NM, class F>
__device__ __forceinline__ void row_filter(const Win& win, F map_of, float (*out)[kS][kT]) {
  for (int it = threadIdx.x; it < kS2 * (kT / 4); it += blockDim.x) {
    const int rp = it / (kT / 4), c0 = (it - rp * (kT / 4)) * 4;
    float2 a[4][NM];
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int m = 0; m < NM; ++m) a[o][m] = f2(0.f);
#pragma unroll
    for (int j = 0; j < 4 + 2 * kR; ++j) {
      float2 v[NM];
      map_of(rp, c0 + j, v);
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int k = j - o;
        if (k >= 0 && k <= 2 * kR) {
          const float2 wk = win.w[k];
#pragma unroll
          for (int m = 0; m < NM; ++m) a[o][m] = fma2(wk, v[m], a[o][m]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        out[m][2 * rp][c0 + o] = a[o][m].x;
        out[m][2 * rp + 1][c0 + o] = a[o][m].y;
      }
  }
}

// Column filter: thread t covers columns (2 cp, 2 cp + 1) as one packed pair
// and rows 2 rg, 2 rg + 1 of the tile (cp = t % 16, rg = t / 16).
template <int NM>
__device__ __forceinline__ void col_filter(const Win& win, float (*in)[kS][kT], float2 (*res)[NM]) {
  const int c = 2 * (threadIdx.x & 15), r0 = 2 * (threadIdx.x >> 4);
#pragma unroll
  for (int o = 0; o < 2; ++o)
#pragma unroll
    for (int m = 0; m < NM; ++m) res[o][m] = f2(0.f);
#pragma unroll
  for (int i = 0; i < 2 + 2 * kR; ++i) {
    float2 v[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) v[m] = *reinterpret_cast<const float2*>(&in[m][r0 + i][c]);
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int k = i - o;
      if (k >= 0 && k <= 2 * kR) {
        const float2 wk = win.w[k];
#pragma unroll
        for (int m = 0; m < NM; ++m) res[o][m] = fma2(wk, v[m], res[o][m]);
      }
    }
  }
}

}  // namespace

// Forward: SSIM at every pixel, the view's loss, and the derivative maps
//   D1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy, D2 = dS/ds_xx, D3 = dS/ds_xy
// (S depends on x through the window sums G*x, G*x^2 and G*(x y)).
// 256 threads per 32 x 32 tile.
__global__ void __launch_bounds__(256, 4) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  int H, int W, Win win, float* __restrict__ dmaps,
                                                  float* __restrict__ ssim_sum) {
  __shared__ float2 s_x[kS2][kS], s_y[kS2][kS];
  __shared__ __align__(16) float s_h[4][kS][kT];
  __shared__ float s_red[8];
  const int tiles_x = (W + kT - 1) / kT;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;  // view * 3 + channel
  const int64_t HW = (int64_t)H * W;
  const int x0 = tx * kT - kR, y0 = ty * kT - kR;
  stage_pairs(img + plane * HW, H, W, x0, y0, s_x);
  stage_pairs(tgt + plane * HW, H, W, x0, y0, s_y);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  // window sums of x, y, x^2 + y^2, x y: SSIM takes the two variances only as
  // their sum, so their second moments are filtered together
  row_filter<4>(win, [&](int rp, int c, float2* v) {
    const float2 xv = s_x[rp][c], yv = s_y[rp][c];
    v[0] = xv; v[1] = yv; v[2] = fma2(xv, xv, mul2(yv, yv)); v[3] = mul2(xv, yv);
  }, s_h);
  __syncthreads();
  float2 m[2][4];
  col_filter<4>(win, s_h, m);
  float local = 0.f;
  const int c = 2 * (threadIdx.x & 15), r0 = 2 * (threadIdx.x >> 4);
  float* d = dmaps + (int64_t)plane * 3 * HW;
#pragma unroll
  for (int o = 0; o < 2; ++o)
#pragma unroll
    for (int hx = 0; hx < 2; ++hx) {
      const int gy = ty * kT + r0 + o, gx = tx * kT + c + hx;
      if (gy >= H || gx >= W) continue;
      const float mx = hx ? m[o][0].y : m[o][0].x, my = hx ? m[o][1].y : m[o][1].x;
      const float ess = hx ? m[o][2].y : m[o][2].x;  // window sum of x^2 + y^2
      const float exy = hx ? m[o][3].y : m[o][3].x;
      const float sxy = exy - mx * my;
      const float a1 = 2.f * mx * my + kC1, a2 = 2.f * sxy + kC2;
      const float b1 = mx * mx + my * my + kC1, b2 = ess - mx * mx - my * my + kC2;  // s_xx + s_yy + C2
      const float ib = 1.f / (b1 * b2);
      const float sv = a1 * a2 * ib;
      const float ds_dmx = 2.f * my * a2 * ib - sv * 2.f * mx / b1;
      const float ds_dsxx = -sv / b2;
      const float ds_dsxy = 2.f * a1 * ib;
      const int64_t p = (int64_t)gy * W + gx;
      d[p] = ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy;
      d[HW + p] = ds_dsxx;
      d[2 * HW + p] = ds_dsxy;
      local += sv;
    }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += s_red[w];
    atomicAdd(ssim_sum + plane / 3, t);
  }
}

// Backward: dD/dx = -(G*D1 + 2 x G*D2 + y G*D3) / (3 H W), added (times the
// weight) to dl_dimg; the window is symmetric, so the adjoint filter is the
// same filter.
__global__ void __launch_bounds__(256) k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  int H, int W, Win win, const float* __restrict__ dmaps,
                                                  float scale, float* __restrict__ dl_dimg) {
  __shared__ float2 s_d[3][kS2][kS];
  __shared__ __align__(16) float s_h[3][kS][kT];
  const int tiles_x = (W + kT - 1) / kT;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;
  const int64_t HW = (int64_t)H * W;
  const float* d = dmaps + (int64_t)plane * 3 * HW;
  const int x0 = tx * kT - kR, y0 = ty * kT - kR;
#pragma unroll
  for (int q = 0; q < 3; ++q) stage_pairs(d + q * HW, H, W, x0, y0, s_d[q]);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  row_filter<3>(win, [&](int rp, int c, float2* v) {
    v[0] = s_d[0][rp][c]; v[1] = s_d[1][rp][c]; v[2] = s_d[2][rp][c];
  }, s_h);
  __syncthreads();
  float2 m[2][3];
  col_filter<3>(win, s_h, m);
  const float* x = img + plane * HW;
  const float* y = tgt + plane * HW;
  float* out = dl_dimg + plane * HW;
  const int c = 2 * (threadIdx.x & 15), r0 = 2 * (threadIdx.x >> 4);
#pragma unroll
  for (int o = 0; o < 2; ++o)
#pragma unroll
    for (int hx = 0; hx < 2; ++hx) {
      const int gy = ty * kT + r0 + o, gx = tx * kT + c + hx;
      if (gy >= H || gx >= W) continue;
      const int64_t p = (int64_t)gy * W + gx;
      const float s0 = hx ? m[o][0].y : m[o][0].x, s1 = hx ? m[o][1].y : m[o][1].x;
      const float s2 = hx ? m[o][2].y : m[o][2].x;
      out[p] += scale * (s0 + 2.f * x[p] * s1 + y[p] * s2);
    }
}

__global__ void k_ssim_loss(const float* __restrict__ ssim_sum, int V, float n, float weight, float* __restrict__ loss) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) loss[v] += weight * (1.f - ssim_sum[v] / n);
}

size_t dssim_scratch_bytes(int V, int H, int W) {
  // three derivative maps per channel plane, then one float per view (SSIM sums)
  return (size_t)V * 3 * 3 * H * W * sizeof(float) + 256 + (size_t)V * sizeof(float);
}

cudaError_t launch_dssim(const float* img, const float* tgt, int V, int H, int W, float weight, float* loss,
                         float* dl_dimg, void* scratch, cudaStream_t st) {
  Win win;
  double g[2 * kR + 1], sum = 0.0;
  for (int k = 0; k <= 2 * kR; ++k) {
    const double d = k - kR;
    g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += g[k];
  }
  for (int k = 0; k <= 2 * kR; ++k) win.w[k] = make_float2((float)(g[k] / sum), (float)(g[k] / sum));
  float* dmaps = static_cast<float*>(scratch);
  float* ssim_sum = reinterpret_cast<float*>(static_cast<char*>(scratch) +
                                             (((size_t)V * 9 * H * W * sizeof(float) + 255) / 256) * 256);
  cudaError_t err = cudaMemsetAsync(ssim_sum, 0, (size_t)V * sizeof(float), st);
  if (err != cudaSuccess) return err;
  const int tiles = ((W + kT - 1) / kT) * ((H + kT - 1) / kT);
  const dim3 grid((unsigned)tiles, (unsigned)(3 * V));
  trace_begin(kKSsimFwd, st);
  k_ssim_fwd<<<grid, 256, 0, st>>>(img, tgt, H, W, win, dmaps, ssim_sum);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (loss) {
    k_ssim_loss<<<(V + 127) / 128, 128, 0, st>>>(ssim_sum, V, 3.f * (float)H * (float)W, weight, loss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (dl_dimg) {
    trace_begin(kKSsimBwd, st);
    k_ssim_bwd<<<grid, 256, 0, st>>>(img, tgt, H, W, win, dmaps, -weight / (3.f * (float)H * (float)W), dl_dimg);
    trace_end(st);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace gsb
