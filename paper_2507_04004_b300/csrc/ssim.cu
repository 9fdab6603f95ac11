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
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Win {
  float w[2 * kR + 1];  // normalised 1D Gaussian; the 2D window is its outer product
};

// Row pass over the staged block: out[r][c] = sum_k w[k] in[r][c + k] for
// the kS rows and kT output columns, for NM maps at once.
template <int NM>
__device__ __forceinline__ void row_pass(const Win& win, float (*in)[kS][kS], float (*out)[kS][kT]) {
  for (int i = threadIdx.x; i < kS * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(win.w[k], in[m][r][c + k], acc);
      out[m][r][c] = acc;
    }
  }
}

}  // namespace

// Forward: SSIM at every pixel, the view's loss, and the derivative maps
//   D1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy, D2 = dS/ds_xx, D3 = dS/ds_xy
// (S depends on x through the window sums G*x, G*x^2 and G*(x y)).
__global__ void __launch_bounds__(256) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  int H, int W, Win win, float* __restrict__ dmaps,
                                                  float* __restrict__ ssim_sum) {
  __shared__ float s_in[2][kS][kS];
  __shared__ float s_h[5][kS][kT];
  __shared__ float s_red[8];
  const int tiles_x = (W + kT - 1) / kT;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;  // view * 3 + channel
  const int64_t HW = (int64_t)H * W;
  const float* x = img + plane * HW;
  const float* y = tgt + plane * HW;
  const int x0 = tx * kT - kR, y0 = ty * kT - kR;
  for (int i = threadIdx.x; i < kS * kS; i += blockDim.x) {
    const int r = i / kS, c = i - r * kS;
    const int gy = y0 + r, gx = x0 + c;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    s_in[0][r][c] = in ? x[(int64_t)gy * W + gx] : 0.f;
    s_in[1][r][c] = in ? y[(int64_t)gy * W + gx] : 0.f;
  }
  __syncthreads();
  // row pass of x, y, x^2, y^2, x y
  for (int i = threadIdx.x; i < kS * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float xv = s_in[0][r][c + k], yv = s_in[1][r][c + k], w = win.w[k];
      a[0] = fmaf(w, xv, a[0]);
      a[1] = fmaf(w, yv, a[1]);
      a[2] = fmaf(w, xv * xv, a[2]);
      a[3] = fmaf(w, yv * yv, a[3]);
      a[4] = fmaf(w, xv * yv, a[4]);
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) s_h[m][r][c] = a[m];
  }
  __syncthreads();
  // column pass and the per-pixel SSIM terms
  float local = 0.f;
  for (int i = threadIdx.x; i < kT * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    const int gy = ty * kT + r, gx = tx * kT + c;
    if (gy >= H || gx >= W) continue;
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float w = win.w[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] = fmaf(w, s_h[q][r + k][c], m[q]);
    }
    const float mx = m[0], my = m[1];
    const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
    const float a1 = 2.f * mx * my + kC1, a2 = 2.f * sxy + kC2;
    const float b1 = mx * mx + my * my + kC1, b2 = sxx + syy + kC2;
    const float ib = 1.f / (b1 * b2);
    const float s = a1 * a2 * ib;
    const float ds_dmx = 2.f * my * a2 * ib - s * 2.f * mx / b1;
    const float ds_dsxx = -s / b2;
    const float ds_dsxy = 2.f * a1 * ib;
    const int64_t p = (int64_t)gy * W + gx;
    float* d = dmaps + (int64_t)plane * 3 * HW;
    d[p] = ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy;
    d[HW + p] = ds_dsxx;
    d[2 * HW + p] = ds_dsxy;
    local += s;
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
  __shared__ float s_in[3][kS][kS];
  __shared__ float s_h[3][kS][kT];
  const int tiles_x = (W + kT - 1) / kT;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;
  const int64_t HW = (int64_t)H * W;
  const float* d = dmaps + (int64_t)plane * 3 * HW;
  const int x0 = tx * kT - kR, y0 = ty * kT - kR;
  for (int i = threadIdx.x; i < kS * kS; i += blockDim.x) {
    const int r = i / kS, c = i - r * kS;
    const int gy = y0 + r, gx = x0 + c;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const int64_t p = (int64_t)gy * W + gx;
#pragma unroll
    for (int m = 0; m < 3; ++m) s_in[m][r][c] = in ? d[m * HW + p] : 0.f;
  }
  __syncthreads();
  row_pass<3>(win, s_in, s_h);
  __syncthreads();
  const float* x = img + plane * HW;
  const float* y = tgt + plane * HW;
  float* out = dl_dimg + plane * HW;
  for (int i = threadIdx.x; i < kT * kT; i += blockDim.x) {
    const int r = i / kT, c = i - r * kT;
    const int gy = ty * kT + r, gx = tx * kT + c;
    if (gy >= H || gx >= W) continue;
    float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float w = win.w[k];
#pragma unroll
      for (int q = 0; q < 3; ++q) m[q] = fmaf(w, s_h[q][r + k][c], m[q]);
    }
    const int64_t p = (int64_t)gy * W + gx;
    out[p] += scale * (m[0] + 2.f * x[p] * m[1] + y[p] * m[2]);
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
  for (int k = 0; k <= 2 * kR; ++k) win.w[k] = (float)(g[k] / sum);
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
