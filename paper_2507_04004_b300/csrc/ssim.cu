// D-SSIM term of the mapping loss (Sec. "Map Optimization") and of the
// tracking loss (Eq. tracking_loss, Sec. "Camera Factor (Option 2)"), which the
// paper takes from 3D Gaussian Splatting: per channel, SSIM of Wang et al.
// under an 11 x 11 Gaussian window (sigma 1.5, zero padding at the borders,
// C1 = 0.01^2, C2 = 0.03^2) and D = 1 - mean SSIM over a view.  Sec.
// "Additional Strategies" (c) computes it with separable Gaussian filters;
// so does this file.  Each CTA owns a 48-wide, 32-tall output tile of one
// channel plane:
//   1. the tile's inputs with their 5-pixel halo arrive in shared memory as
//      one TMA box per plane (zero outside the image, filled by the copy
//      engine), or by cp.async where the image rows are not 16-byte strided;
//   2. the vertical filter runs down the staged columns on horizontal pixel
//      pairs (packed FP32x2) and leaves its sums interleaved by row pairs;
//   3. the horizontal filter runs along those on vertical pixel pairs, and
//      the same thread finishes its 8 pixels (SSIM and its derivative maps
//      in the forward pass, the image gradient in the backward pass, whose
//      per-pixel operands a second TMA copy brings in meanwhile).
#include <cmath>
#include <cstring>

#include <cuda.h>

#include "gs_internal.h"

namespace gsb {

namespace {

constexpr int kTW = 48;            // output tile width
constexpr int kTH = 32;            // output tile height
constexpr int kR = 5;              // window radius
constexpr int kThreads = 256;
// Staged box: columns tx*48 - 8 .. tx*48 + 55 (the left edge on a 16-byte
// boundary, as TMA requires; the filters use columns 3 .. 60 of the box),
// rows ty*32 - 5 .. ty*32 + 36.
constexpr int kBX = 64;
constexpr int kBY = kTH + 2 * kR;  // 42
constexpr int kBXOff = 8;
// Vertical filter: lanes 0..29 of warp w take the column pair (2 + 2 lane,
// 3 + 2 lane) of the box and output rows 4w .. 4w + 3.
constexpr int kVPairs = 30;
constexpr int kVRows = kTH / (kThreads / 32);  // 4
// Its sums: hp[m][i][k] = (row 2i, row 2i + 1) at box column k + 2; the odd
// row stride keeps the horizontal filter's loads free of bank conflicts.
constexpr int kHP = 61;
// Horizontal filter: threads 0..191, each one row pair i and the output
// columns 4q .. 4q + 3 (see hitem).
constexpr int kHItems = (kTH / 2) * (kTW / 4);  // 192
// Output tiles ([kTH][kTW] per map, dense: the TMA store box) and the
// backward's operand tiles (x, y, dl_dimg over the output tile).
constexpr int kOutFloats = kTH * kTW;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;
constexpr uint64_t kWaitNs = 1000000000ull;  // bound on a TMA wait (1 s)

static_assert(kVRows == 4 && kTH == 32 && kTW == 48, "tile shape");
static_assert(kBX >= kBXOff + kTW + kR && 2 + 2 * kVPairs <= kBX, "box covers the window");
static_assert(kHP >= 2 * kVPairs && 4 * (kTW / 4 - 1) + 1 + 13 < 2 * kVPairs, "horizontal filter reads");

constexpr size_t kPlaneBytes = (size_t)kBX * kBY * sizeof(float);  // 10752, a multiple of 128
constexpr size_t kHpBytes = (size_t)(kTH / 2) * kHP * sizeof(float2);
constexpr size_t kEpBytes = (size_t)kOutFloats * sizeof(float);
// forward: staged x, y | hp[4] | reduction | barrier
constexpr size_t kFwdHp = 2 * kPlaneBytes;
constexpr size_t kFwdRed = kFwdHp + 4 * kHpBytes;
constexpr size_t kFwdBar = (kFwdRed + 8 * sizeof(float) + 15) / 16 * 16;
constexpr size_t kFwdSmem = kFwdBar + 16 + 128;  // + alignment slack of the dynamic base
// backward: staged D1, D2, D3 (then x, y, dl_dimg in their place) | hp[3] | barriers
constexpr size_t kBwdHp = 3 * kPlaneBytes;
constexpr size_t kBwdBar = kBwdHp + 3 * kHpBytes;
constexpr size_t kBwdSmem = kBwdBar + 16 + 128;
static_assert(kPlaneBytes % 128 == 0 && kEpBytes % 128 == 0 && 3 * kEpBytes <= 2 * kPlaneBytes, "staging layout");

struct Win {
  // normalised 1D Gaussian (the 2D window is its outer product), each weight
  // twice so that the packed FP32 pair instructions take it as it stands
  float2 w[2 * kR + 1];
};

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for phase `parity` of the barrier; false once kWaitNs has passed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// One box of a [planes][H][W] FP32 tensor map at (x, y, plane) into shared
// memory, completing its bytes on the barrier (out-of-image elements read 0).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// One box of a [planes][H][W] FP32 tensor map into L2 (no shared memory, no
// completion to wait for: a hint).
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

// Order the block's earlier shared-memory accesses (this thread's, and after
// a barrier everyone's) before later async-proxy (TMA) writes to the same bytes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared memory -> one box of a [planes][H][W] FP32 tensor map at (x, y,
// plane) (elements outside the tensor are not written); the issuing thread
// then waits until the copy has read shared memory.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit_and_wait_read() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// 4-byte asynchronous copy into shared memory, zero-filled when `in` is
// false (no global byte is read then; `src` must still be a valid address).
__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(in ? 4 : 0)
               : "memory");
}

// The same box as tma_load_3d, element by element (rows of any stride).
template <int BX, int BY>
__device__ __forceinline__ void copy_box(const float* __restrict__ plane, int H, int W, int gx0, int gy0, float* dst) {
  for (int e = threadIdx.x; e < BX * BY; e += kThreads) {
    const int r = e / BX, s = e - r * BX;
    const int gx = gx0 + s, gy = gy0 + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    cp_async4_zfill(dst + e, in ? plane + (int64_t)gy * W + gx : plane, in);
  }
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// Reciprocal of each half by the hardware approximation (within a few units
// in the last place; the arguments here are at least C1 C2, far from the
// denormal range).
__device__ __forceinline__ float2 rcp2_approx(float2 a) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(a.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(a.y));
  return r;
}

// Horizontal-filter thread t < 192: row pair i and column quad q.  A warp
// takes 8 row pairs x 4 quads, the lane bits (3, 0, 4) giving the row pair
// and (1, 2) the quad; with hp's row stride of 61 its hp loads, and its
// 16-byte accesses to a dense [32][48] tile in the order of tile_rows, are
// free of bank conflicts.
__device__ __forceinline__ void hitem(int t, int& i, int& q) {
  const int w = t >> 5, l = t & 31;
  i = (w & 1) * 8 + (((l >> 3) & 1) | ((l & 1) << 1) | (((l >> 4) & 1) << 2));
  q = (w >> 1) * 4 + ((l >> 1) & 3);
}

// The two rows of row pair i in the order the thread accesses a dense tile:
// lanes with bit 1 of i set take the odd row first.
__device__ __forceinline__ void tile_rows(int i, int& first, int& second) {
  const int sel = (i >> 1) & 1;
  first = 2 * i + sel;
  second = 2 * i + 1 - sel;
}

__device__ __forceinline__ bool aligned16(const float* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Four consecutive pixels of a row from column gx: one 16-byte store where
// all lie in the image and the address allows it, else one by one.
__device__ __forceinline__ void store_row4(float* row, int gx, int W, float a, float b, float c, float d) {
  if (gx + 3 < W && aligned16(row + gx)) {
    *reinterpret_cast<float4*>(row + gx) = make_float4(a, b, c, d);
  } else {
    if (gx < W) row[gx] = a;
    if (gx + 1 < W) row[gx + 1] = b;
    if (gx + 2 < W) row[gx + 2] = c;
    if (gx + 3 < W) row[gx + 3] = d;
  }
}

// ---------------------------------------------------------------------------
// The two filter passes

// Vertical filter of NM maps formed from the staged planes by map_of(row,
// column, v) (v[m] = the maps at that box row for the thread's column pair):
// output rows 4w .. 4w + 3 from box rows 4w .. 4w + 13, into hp.
template <int NM, class F>
__device__ __forceinline__ void vertical_filter(const Win& win, F map_of, float2* __restrict__ hp) {
  const int w = threadIdx.x >> 5, j = threadIdx.x & 31;
  if (j >= kVPairs) return;
  const int col = 2 + 2 * j, r0 = kVRows * w;
  float2 acc[kVRows][NM];
#pragma unroll
  for (int o = 0; o < kVRows; ++o)
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[o][m] = f2(0.f);
#pragma unroll
  for (int i = 0; i < kVRows + 2 * kR; ++i) {
    float2 v[NM];
    map_of(r0 + i, col, v);
#pragma unroll
    for (int o = 0; o < kVRows; ++o) {
      const int k = i - o;
      if (k >= 0 && k <= 2 * kR) {
        const float2 wk = win.w[k];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[o][m] = fma2(wk, v[m], acc[o][m]);
      }
    }
  }
  // (rows 4w, 4w + 1) -> row pair 2w, (4w + 2, 4w + 3) -> 2w + 1.  Of the
  // thread's two columns, lanes with bit 3 clear store the left one first and
  // the others the right one, so each half-warp's stores cover all 32 banks
  // once per instruction.
  const bool swap = (j >> 3) & 1;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    float2* h = hp + (size_t)m * (kTH / 2) * kHP + (size_t)(2 * w) * kHP + 2 * j;
#pragma unroll
    for (int rp = 0; rp < 2; ++rp) {
      const float2 left = make_float2(acc[2 * rp][m].x, acc[2 * rp + 1][m].x);
      const float2 right = make_float2(acc[2 * rp][m].y, acc[2 * rp + 1][m].y);
      h[rp * kHP + (swap ? 1 : 0)] = swap ? right : left;
      h[rp * kHP + (swap ? 0 : 1)] = swap ? left : right;
    }
  }
}

// Horizontal filter of the NM interleaved maps for row pair i and output
// columns 4q .. 4q + 3: res[o][m] = (row 2i, row 2i + 1) at column 4q + o.
template <int NM>
__device__ __forceinline__ void horizontal_filter(const Win& win, const float2* __restrict__ hp, int i, int q,
                                                  float2 (*res)[NM]) {
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int m = 0; m < NM; ++m) res[o][m] = f2(0.f);
  const float2* h = hp + (size_t)i * kHP + 4 * q + 1;
#pragma unroll
  for (int jj = 0; jj < 4 + 2 * kR; ++jj) {
    float2 v[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) v[m] = h[(size_t)m * (kTH / 2) * kHP + jj];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int k = jj - o;
      if (k >= 0 && k <= 2 * kR) {
        const float2 wk = win.w[k];
#pragma unroll
        for (int m = 0; m < NM; ++m) res[o][m] = fma2(wk, v[m], res[o][m]);
      }
    }
  }
}

__device__ __forceinline__ unsigned char* smem_base(unsigned char* raw) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
}

}  // namespace

// Forward: SSIM at every pixel, the view's loss, and the derivative maps
//   D1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy, D2 = dS/ds_xx, D3 = dS/ds_xy
// (S depends on x through the window sums G*x, G*x^2 and G*(x y)), written
// by TMA from output tiles in the dead staging space.  A TMA wait that runs
// out (never expected) adds NaN to the view's SSIM sum.
template <bool TMA>
__global__ void __launch_bounds__(kThreads, 4)
    k_ssim_fwd(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_y,
               const __grid_constant__ CUtensorMap map_d, const float* __restrict__ img,
               const float* __restrict__ tgt, int H, int W, Win win, float* __restrict__ dmaps,
               float* __restrict__ ssim_sum) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sb = smem_base(smem_raw);
  float* sx = reinterpret_cast<float*>(sb);
  float* sy = reinterpret_cast<float*>(sb + kPlaneBytes);
  float* so = sx;  // output tiles D1, D2, D3 once the staged planes are dead
  float2* hp = reinterpret_cast<float2*>(sb + kFwdHp);
  float* red = reinterpret_cast<float*>(sb + kFwdRed);
  const uint32_t bar = smem_u32(sb + kFwdBar);
  const int tiles_x = (W + kTW - 1) / kTW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;  // view * 3 + channel
  const int64_t HW = (int64_t)H * W;
  const int gx0 = tx * kTW - kBXOff, gy0 = ty * kTH - kR;
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(bar);
      mbar_init_fence();
      mbar_expect_tx(bar, 2 * (uint32_t)kPlaneBytes);
      tma_load_3d(smem_u32(sx), &map_x, gx0, gy0, plane, bar);
      tma_load_3d(smem_u32(sy), &map_y, gx0, gy0, plane, bar);
    }
    __syncthreads();  // the barrier's initialisation before anyone waits on it
    if (!__syncthreads_and(mbar_wait(bar, 0))) {
      mbar_wait(bar, 0);  // let copies still in flight land before the block exits
      if (threadIdx.x == 0) atomicAdd(ssim_sum + plane / 3, __int_as_float(0x7fc00000));
      return;
    }
  } else {
    copy_box<kBX, kBY>(img + plane * HW, H, W, gx0, gy0, sx);
    copy_box<kBX, kBY>(tgt + plane * HW, H, W, gx0, gy0, sy);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
  }
  // window sums of x, y, x^2 + y^2, x y: SSIM takes the two variances only as
  // their sum, so their second moments are filtered together
  vertical_filter<4>(win, [&](int r, int c, float2* v) {
    const float2 xv = *reinterpret_cast<const float2*>(sx + r * kBX + c);
    const float2 yv = *reinterpret_cast<const float2*>(sy + r * kBX + c);
    v[0] = xv; v[1] = yv; v[2] = fma2(xv, xv, mul2(yv, yv)); v[3] = mul2(xv, yv);
  }, hp);
  __syncthreads();
  float local = 0.f;
  const int ex0 = tx * kTW, ey0 = ty * kTH;  // output tile origin
  if (threadIdx.x < kHItems) {
    int i, q;
    hitem(threadIdx.x, i, q);
    float2 m[4][4];
    horizontal_filter<4>(win, hp, i, q, m);
    const float2 C1 = f2(kC1), C2 = f2(kC2), two = f2(2.f);
    float2 dd[3][4];  // D1, D2, D3 at (row 2i, row 2i + 1), column 4q + o
    const int gy = ey0 + 2 * i, gx = ex0 + 4 * q;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const float2 mx = m[o][0], my = m[o][1], ess = m[o][2], exy = m[o][3];  // ess: window sum of x^2 + y^2
      const float2 mxy = mul2(mx, my), mm = fma2(mx, mx, mul2(my, my));
      const float2 a1 = fma2(two, mxy, C1), a2 = fma2(two, sub2(exy, mxy), C2);  // 2 mu_x mu_y + C1, 2 s_xy + C2
      const float2 b1 = add2(mm, C1), b2 = add2(sub2(ess, mm), C2);  // mu_x^2 + mu_y^2 + C1, s_xx + s_yy + C2
      const float2 ib = rcp2_approx(mul2(b1, b2));
      const float2 a2ib = mul2(a2, ib);
      const float2 sv = mul2(a1, a2ib);
      const float2 ds_dsxy = mul2(two, mul2(a1, ib));
      const float2 sv_b2 = mul2(sv, mul2(b1, ib));  // S / b2 = -dS/ds_xx
      // dS/dmu_x = 2 mu_y a2 / (b1 b2) - 2 mu_x S / b1, with 1 / b1 = b2 ib
      const float2 ds_dmx = mul2(two, sub2(mul2(my, a2ib), mul2(mx, mul2(sv, mul2(b2, ib)))));
      dd[0][o] = sub2(fma2(mul2(two, mx), sv_b2, ds_dmx), mul2(my, ds_dsxy));
      dd[1][o] = make_float2(-sv_b2.x, -sv_b2.y);
      dd[2][o] = ds_dsxy;
      if (gx + o < W) local += (gy < H ? sv.x : 0.f) + (gy + 1 < H ? sv.y : 0.f);
    }
    if (TMA) {
      int ra, rb;
      tile_rows(i, ra, rb);
      const bool odd_first = ra & 1;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float4 ev = make_float4(dd[k][0].x, dd[k][1].x, dd[k][2].x, dd[k][3].x);
        const float4 od = make_float4(dd[k][0].y, dd[k][1].y, dd[k][2].y, dd[k][3].y);
        *reinterpret_cast<float4*>(so + k * kOutFloats + ra * kTW + 4 * q) = odd_first ? od : ev;
        *reinterpret_cast<float4*>(so + k * kOutFloats + rb * kTW + 4 * q) = odd_first ? ev : od;
      }
    } else {
      float* d = dmaps + (int64_t)plane * 3 * HW;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (gy < H) store_row4(d + k * HW + (int64_t)gy * W, gx, W, dd[k][0].x, dd[k][1].x, dd[k][2].x, dd[k][3].x);
        if (gy + 1 < H)
          store_row4(d + k * HW + (int64_t)(gy + 1) * W, gx, W, dd[k][0].y, dd[k][1].y, dd[k][2].y, dd[k][3].y);
      }
    }
  }
  if (TMA) fence_proxy_async();  // the output tiles, to the copy engine
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (TMA) {
#pragma unroll
      for (int k = 0; k < 3; ++k) tma_store_3d(&map_d, smem_u32(so + k * kOutFloats), ex0, ey0, 3 * plane + k);
    }
    float t = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    atomicAdd(ssim_sum + plane / 3, t);
    if (TMA) tma_store_commit_and_wait_read();
  }
}

// Backward: dD/dx = -(G*D1 + 2 x G*D2 + y G*D3) / (3 H W), added (times the
// weight) to dl_dimg; the window is symmetric, so the adjoint filter is the
// same filter.  x, y and dl_dimg over the tile come in by TMA, the updated
// dl_dimg goes out by TMA from the same shared memory.  A TMA wait that runs
// out (never expected) leaves NaN in the tile's dl_dimg.
template <bool TMA>
__global__ void __launch_bounds__(kThreads, 4)
    k_ssim_bwd(const __grid_constant__ CUtensorMap map_d, const __grid_constant__ CUtensorMap map_x,
               const __grid_constant__ CUtensorMap map_y, const __grid_constant__ CUtensorMap map_dl,
               const float* __restrict__ img, const float* __restrict__ tgt, int H, int W, Win win,
               const float* __restrict__ dmaps, float scale, float* __restrict__ dl_dimg) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sb = smem_base(smem_raw);
  float* sd = reinterpret_cast<float*>(sb);  // D1, D2, D3 boxes; then x, y, dl_dimg over the tile
  float2* hp = reinterpret_cast<float2*>(sb + kBwdHp);
  const uint32_t bar0 = smem_u32(sb + kBwdBar), bar1 = bar0 + 8;
  const int tiles_x = (W + kTW - 1) / kTW;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int plane = blockIdx.y;
  const int64_t HW = (int64_t)H * W;
  const float* d = dmaps + (int64_t)plane * 3 * HW;
  float* out = dl_dimg + plane * HW;
  const int gx0 = tx * kTW - kBXOff, gy0 = ty * kTH - kR;
  const int ex0 = tx * kTW, ey0 = ty * kTH;  // output tile origin
  float* ep = sd;                            // operand tiles [3][kTH][kTW]
  constexpr int kPlaneFloats = (int)(kPlaneBytes / sizeof(float));
  bool ok = true;
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(bar0);
      mbar_init(bar1);
      mbar_init_fence();
      mbar_expect_tx(bar0, 3 * (uint32_t)kPlaneBytes);
#pragma unroll
      for (int k = 0; k < 3; ++k) tma_load_3d(smem_u32(sd + k * kPlaneFloats), &map_d, gx0, gy0, 3 * plane + k, bar0);
      // the epilogue's x, y and dl_dimg tiles, loaded after the vertical
      // filter, are pulled into L2 now
      tma_prefetch_l2_3d(&map_x, ex0, ey0, plane);
      tma_prefetch_l2_3d(&map_y, ex0, ey0, plane);
      tma_prefetch_l2_3d(&map_dl, ex0, ey0, plane);
    }
    __syncthreads();
    ok = __syncthreads_and(mbar_wait(bar0, 0));
    if (!ok) mbar_wait(bar0, 0);
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) copy_box<kBX, kBY>(d + k * HW, H, W, gx0, gy0, sd + k * kPlaneFloats);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
  }
  if (ok) {
    vertical_filter<3>(win, [&](int r, int c, float2* v) {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = *reinterpret_cast<const float2*>(sd + k * kPlaneFloats + r * kBX + c);
    }, hp);
  }
  __syncthreads();
  // the staged maps are dead: fetch x, y and dl_dimg over the output tile
  // into their place while the horizontal filter runs
  if (TMA) {
    if (ok && threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar1, 3 * (uint32_t)kEpBytes);
      tma_load_3d(smem_u32(ep), &map_x, ex0, ey0, plane, bar1);
      tma_load_3d(smem_u32(ep + kOutFloats), &map_y, ex0, ey0, plane, bar1);
      tma_load_3d(smem_u32(ep + 2 * kOutFloats), &map_dl, ex0, ey0, plane, bar1);
    }
  } else {
    copy_box<kTW, kTH>(img + plane * HW, H, W, ex0, ey0, ep);
    copy_box<kTW, kTH>(tgt + plane * HW, H, W, ex0, ey0, ep + kOutFloats);
    copy_box<kTW, kTH>(out, H, W, ex0, ey0, ep + 2 * kOutFloats);
    cp_async_commit();
  }
  int i, q;
  hitem(threadIdx.x, i, q);
  float2 m[4][3];
  if (threadIdx.x < kHItems && ok) horizontal_filter<3>(win, hp, i, q, m);
  if (TMA) {
    if (ok) {
      ok = __syncthreads_and(mbar_wait(bar1, 0));
      if (!ok) mbar_wait(bar1, 0);
    }
  } else {
    cp_async_wait_all();
    __syncthreads();
  }
  const int gy = ey0 + 2 * i, gx = ex0 + 4 * q;
  if (!ok) {
    if (threadIdx.x < kHItems) {
      const float nan = __int_as_float(0x7fc00000);
      if (gy < H) store_row4(out + (int64_t)gy * W, gx, W, nan, nan, nan, nan);
      if (gy + 1 < H) store_row4(out + (int64_t)(gy + 1) * W, gx, W, nan, nan, nan, nan);
    }
    return;
  }
  if (threadIdx.x < kHItems) {
    // operands of rows 2i, 2i + 1, columns 4q .. 4q + 3 (zero outside the image)
    int ra, rb;
    tile_rows(i, ra, rb);
    const bool odd_first = ra & 1;
    float4 v[3][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(ep + k * kOutFloats + ra * kTW + 4 * q);
      const float4 b = *reinterpret_cast<const float4*>(ep + k * kOutFloats + rb * kTW + 4 * q);
      v[k][0] = odd_first ? b : a;  // row 2i
      v[k][1] = odd_first ? a : b;  // row 2i + 1
    }
    const float2 sc = f2(scale);
    float g[2][4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      auto col = [&](const float4& r) { return o == 0 ? r.x : o == 1 ? r.y : o == 2 ? r.z : r.w; };
      const float2 xv = make_float2(col(v[0][0]), col(v[0][1])), yv = make_float2(col(v[1][0]), col(v[1][1]));
      const float2 r = fma2(sc, fma2(add2(xv, xv), m[o][1], fma2(yv, m[o][2], m[o][0])),
                            make_float2(col(v[2][0]), col(v[2][1])));
      g[0][o] = r.x;
      g[1][o] = r.y;
    }
    if (TMA) {
      // the updated dl_dimg in place of the loaded one (each element read and
      // written by this thread only), rows in the same order
      const float4 ev = make_float4(g[0][0], g[0][1], g[0][2], g[0][3]);
      const float4 od = make_float4(g[1][0], g[1][1], g[1][2], g[1][3]);
      *reinterpret_cast<float4*>(ep + 2 * kOutFloats + ra * kTW + 4 * q) = odd_first ? od : ev;
      *reinterpret_cast<float4*>(ep + 2 * kOutFloats + rb * kTW + 4 * q) = odd_first ? ev : od;
    } else {
      if (gy < H) store_row4(out + (int64_t)gy * W, gx, W, g[0][0], g[0][1], g[0][2], g[0][3]);
      if (gy + 1 < H) store_row4(out + (int64_t)(gy + 1) * W, gx, W, g[1][0], g[1][1], g[1][2], g[1][3]);
    }
  }
  if (TMA) {
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_3d(&map_dl, smem_u32(ep + 2 * kOutFloats), ex0, ey0, plane);
      tma_store_commit_and_wait_read();
    }
  }
}

__global__ void k_ssim_loss(const float* __restrict__ ssim_sum, int V, float n, float weight, float* __restrict__ loss) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) loss[v] += weight * (1.f - ssim_sum[v] / n);
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null when unavailable.
EncodeTiled encoder() {
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<EncodeTiled>(nullptr);
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of `planes` FP32 planes of H x W at `base`, boxes of bx x by x 1
// (zero fill outside).  Needs W % 4 == 0 and a 16-byte aligned base.
bool encode_planes(CUtensorMap* map, const float* base, int planes, int H, int W, int bx, int by) {
  const EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)W * sizeof(float), (cuuint64_t)W * H * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16_host(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

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
  // TMA needs 16-byte row strides and bases; other shapes stage by cp.async
  // and store directly
  CUtensorMap mx, my, md, mdo, ex, ey, el;
  for (CUtensorMap* mp : {&mx, &my, &md, &mdo, &ex, &ey, &el}) std::memset(mp, 0, sizeof(CUtensorMap));
  const bool tma = W % 4 == 0 && aligned16_host(img) && aligned16_host(tgt) && aligned16_host(dmaps) &&
                   (!dl_dimg || aligned16_host(dl_dimg)) && encode_planes(&mx, img, 3 * V, H, W, kBX, kBY) &&
                   encode_planes(&my, tgt, 3 * V, H, W, kBX, kBY) && encode_planes(&md, dmaps, 9 * V, H, W, kBX, kBY) &&
                   encode_planes(&mdo, dmaps, 9 * V, H, W, kTW, kTH) &&
                   encode_planes(&ex, img, 3 * V, H, W, kTW, kTH) && encode_planes(&ey, tgt, 3 * V, H, W, kTW, kTH) &&
                   (!dl_dimg || encode_planes(&el, dl_dimg, 3 * V, H, W, kTW, kTH));
  const int tiles = ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
  const dim3 grid((unsigned)tiles, (unsigned)(3 * V));
  auto fwd = tma ? k_ssim_fwd<true> : k_ssim_fwd<false>;
  auto bwd = tma ? k_ssim_bwd<true> : k_ssim_bwd<false>;
  if ((err = cudaFuncSetAttribute(fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem)) != cudaSuccess)
    return err;
  if ((err = cudaFuncSetAttribute(bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem)) != cudaSuccess)
    return err;
  // four CTAs per SM need the largest shared-memory carveout
  if ((err = cudaFuncSetAttribute(fwd, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return err;
  if ((err = cudaFuncSetAttribute(bwd, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return err;
  trace_begin(kKSsimFwd, st);
  fwd<<<grid, kThreads, kFwdSmem, st>>>(mx, my, mdo, img, tgt, H, W, win, dmaps, ssim_sum);
  trace_end(st);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (loss) {
    k_ssim_loss<<<(V + 127) / 128, 128, 0, st>>>(ssim_sum, V, 3.f * (float)H * (float)W, weight, loss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (dl_dimg) {
    trace_begin(kKSsimBwd, st);
    bwd<<<grid, kThreads, kBwdSmem, st>>>(md, ex, ey, el, img, tgt, H, W, win, dmaps,
                                          -weight / (3.f * (float)H * (float)W), dl_dimg);
    trace_end(st);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace gsb
