// Camera tracking against a fixed map (Sec. "Camera Factor (Option 2)"): the
// pose of each frame is optimised for N_t Adam iterations on the loss of
// Eq. tracking_loss while the Gaussians stay fixed.  The pose is
// parameterised as the right perturbation T_v = T0_v Exp(xi_v) of an initial
// world-to-camera transform, xi = (rho, theta), the same convention as the
// pose gradient of Eq. 3dgs_jacobi in gs_render_bwd, so that gradient is the
// Adam gradient as it stands.  Two small kernels: apply the perturbation to
// the camera batch, and the Adam step on every view's xi.
#include <cmath>

#include "gs_internal.h"

namespace gsb {

// Exp of a twist xi = (rho, theta): R = exp([theta]x) (Rodrigues), t = V rho,
// V = I + (1 - cos p)/p^2 [theta]x + (p - sin p)/p^3 [theta]x^2, p = |theta|;
// series for small p.  Writes cams_out[v] = cams0[v] * Exp(xi[v]):
// R = R0 R_xi, t = R0 V rho + t0, intrinsics copied.
__global__ void k_pose_apply(const gs_camera* __restrict__ cams0, const float* __restrict__ xi, int V,
                             gs_camera* __restrict__ cams_out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float* x = xi + 6 * v;
  const float r0 = x[0], r1 = x[1], r2 = x[2], w0 = x[3], w1 = x[4], w2 = x[5];
  const float p2 = w0 * w0 + w1 * w1 + w2 * w2;
  float a, b, c;  // sin p / p, (1 - cos p) / p^2, (p - sin p) / p^3
  if (p2 < 1e-8f) {
    a = 1.f - p2 / 6.f;
    b = 0.5f - p2 / 24.f;
    c = 1.f / 6.f - p2 / 120.f;
  } else {
    const float p = sqrtf(p2);
    const float s = sinf(p), co = cosf(p);
    a = s / p;
    b = (1.f - co) / p2;
    c = (p - s) / (p2 * p);
  }
  // [w]x and [w]x^2
  const float K[3][3] = {{0.f, -w2, w1}, {w2, 0.f, -w0}, {-w1, w0, 0.f}};
  float K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[i][j] = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
  float R[3][3], Vm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const float id = i == j ? 1.f : 0.f;
      R[i][j] = id + a * K[i][j] + b * K2[i][j];
      Vm[i][j] = id + b * K[i][j] + c * K2[i][j];
    }
  const float tx[3] = {Vm[0][0] * r0 + Vm[0][1] * r1 + Vm[0][2] * r2, Vm[1][0] * r0 + Vm[1][1] * r1 + Vm[1][2] * r2,
                       Vm[2][0] * r0 + Vm[2][1] * r1 + Vm[2][2] * r2};
  const gs_camera c0 = cams0[v];
  gs_camera out = c0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      out.R[3 * i + j] = c0.R[3 * i + 0] * R[0][j] + c0.R[3 * i + 1] * R[1][j] + c0.R[3 * i + 2] * R[2][j];
    out.t[i] = c0.R[3 * i + 0] * tx[0] + c0.R[3 * i + 1] * tx[1] + c0.R[3 * i + 2] * tx[2] + c0.t[i];
  }
  cams_out[v] = out;
}

// One Adam step (Kingma and Ba) on every view's xi with per-component
// learning rates; the step counter lives on the device so that a captured
// loop of iterations replays correctly.  The gradient is cleared for the next
// backward pass (which adds to it).  With loss / best_loss / best_xi given,
// the iterate whose loss (evaluated before this step) is the lowest so far is
// kept per view.
__global__ void k_adam_pose(float* __restrict__ xi, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ s, int32_t* __restrict__ step, int V, gs_adam_config hp,
                            const float* __restrict__ loss, float* __restrict__ best_loss,
                            float* __restrict__ best_xi) {
  const int t = *step + 1;
  const bool keep = loss && best_loss && best_xi;
  for (int i = threadIdx.x; i < 6 * V; i += blockDim.x) {
    if (keep && loss[i / 6] < best_loss[i / 6]) best_xi[i] = xi[i];
  }
  __syncthreads();  // every component has compared against the old best before it changes
  if (keep)
    for (int v = threadIdx.x; v < V; v += blockDim.x)
      if (loss[v] < best_loss[v]) best_loss[v] = loss[v];
  for (int i = threadIdx.x; i < 6 * V; i += blockDim.x) {
    const float g = grad[i];
    const float mi = hp.beta1 * m[i] + (1.f - hp.beta1) * g;
    const float si = hp.beta2 * s[i] + (1.f - hp.beta2) * g * g;
    m[i] = mi;
    s[i] = si;
    const float mh = mi / (1.f - powf(hp.beta1, (float)t));
    const float sh = si / (1.f - powf(hp.beta2, (float)t));
    xi[i] -= hp.lr[i % 6] * mh / (sqrtf(sh) + hp.eps);
    grad[i] = 0.f;
  }
  __syncthreads();  // one block: every thread has read *step before it advances
  if (threadIdx.x == 0) *step = t;
}

// Photometric residual of camera factor option 2 (Eq. map_optimize_pose):
// r = Log(T(t) T~^-1) with T(t) and T~ camera-to-world.  The library's
// cameras are world-to-camera, A = T(t)^-1 and B = T~^-1, so r = Log(A^-1 B),
// the twist (rho, theta) with Exp(r) = A^-1 B: B = A Exp(r), the convention of
// k_pose_apply (for B = T0 Exp(xi) and A = T0, r = xi).
//   rotation: theta = p u from the unit quaternion (w, v) of R = R_A^T R_B
//     (largest-pivot extraction), p = 2 atan2(|v|, w) in [0, pi] with w >= 0
//     (well conditioned at 0 and at pi, unlike acos of the trace);
//   translation: rho = V^-1 t, t = R_A^T (t_B - t_A),
//     V^-1 = I - 1/2 [theta]x + c [theta]x^2,
//     c = (1 - (p/2) cot(p/2)) / p^2, by its series 1/12 + p^2/720 + p^4/30240
//     below p = 0.5 (the closed form cancels there).
__global__ void k_pose_residual(const gs_camera* __restrict__ cams_a, const gs_camera* __restrict__ cams_b, int V,
                                float* __restrict__ r) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const gs_camera A = cams_a[v], B = cams_b[v];
  float R[3][3], t[3];
  const float dt[3] = {B.t[0] - A.t[0], B.t[1] - A.t[1], B.t[2] - A.t[2]};
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      R[i][j] = A.R[0 * 3 + i] * B.R[0 * 3 + j] + A.R[1 * 3 + i] * B.R[1 * 3 + j] + A.R[2 * 3 + i] * B.R[2 * 3 + j];
    t[i] = A.R[0 * 3 + i] * dt[0] + A.R[1 * 3 + i] * dt[1] + A.R[2 * 3 + i] * dt[2];
  }
  // quaternion (qw, qx, qy, qz) of R, pivot on the largest of 4 qw^2, 4 qx^2, 4 qy^2, 4 qz^2
  const float tr = R[0][0] + R[1][1] + R[2][2];
  float qw, qx, qy, qz;
  if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + tr, 1e-30f));  // 4 qw
    qw = 0.25f * s; qx = (R[2][1] - R[1][2]) / s; qy = (R[0][2] - R[2][0]) / s; qz = (R[1][0] - R[0][1]) / s;
  } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[0][0] - R[1][1] - R[2][2], 1e-30f));  // 4 qx
    qw = (R[2][1] - R[1][2]) / s; qx = 0.25f * s; qy = (R[0][1] + R[1][0]) / s; qz = (R[0][2] + R[2][0]) / s;
  } else if (R[1][1] >= R[2][2]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[1][1] - R[0][0] - R[2][2], 1e-30f));  // 4 qy
    qw = (R[0][2] - R[2][0]) / s; qx = (R[0][1] + R[1][0]) / s; qy = 0.25f * s; qz = (R[1][2] + R[2][1]) / s;
  } else {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[2][2] - R[0][0] - R[1][1], 1e-30f));  // 4 qz
    qw = (R[1][0] - R[0][1]) / s; qx = (R[0][2] + R[2][0]) / s; qy = (R[1][2] + R[2][1]) / s; qz = 0.25f * s;
  }
  if (qw < 0.f) { qw = -qw; qx = -qx; qy = -qy; qz = -qz; }
  const float sv = sqrtf(qx * qx + qy * qy + qz * qz);
  const float p = 2.f * atan2f(sv, qw);
  // theta = p v / |v|; as |v| -> 0, p / |v| -> 2 / qw
  const float k = sv > 0.f ? p / sv : 2.f / fmaxf(qw, 1e-30f);
  const float w0 = k * qx, w1 = k * qy, w2 = k * qz;
  const float p2 = w0 * w0 + w1 * w1 + w2 * w2;
  float c;
  if (p2 < 0.25f) {
    c = 1.f / 12.f + p2 * (1.f / 720.f + p2 * (1.f / 30240.f));
  } else {
    const float hp = 0.5f * sqrtf(p2);
    c = (1.f - hp * cosf(hp) / sinf(hp)) / p2;
  }
  // V^-1 t = t - 1/2 theta x t + c theta x (theta x t)
  const float cx0 = w1 * t[2] - w2 * t[1], cx1 = w2 * t[0] - w0 * t[2], cx2 = w0 * t[1] - w1 * t[0];
  const float dx0 = w1 * cx2 - w2 * cx1, dx1 = w2 * cx0 - w0 * cx2, dx2 = w0 * cx1 - w1 * cx0;
  float* o = r + 6 * v;
  o[0] = t[0] - 0.5f * cx0 + c * dx0;
  o[1] = t[1] - 0.5f * cx1 + c * dx1;
  o[2] = t[2] - 0.5f * cx2 + c * dx2;
  o[3] = w0;
  o[4] = w1;
  o[5] = w2;
}

cudaError_t launch_pose_residual(const gs_camera* cams_a, const gs_camera* cams_b, int V, float* r, cudaStream_t st) {
  k_pose_residual<<<(V + 63) / 64, 64, 0, st>>>(cams_a, cams_b, V, r);
  return cudaGetLastError();
}

cudaError_t launch_pose_apply(const gs_camera* cams0, const float* xi, int V, gs_camera* cams_out, cudaStream_t st) {
  k_pose_apply<<<(V + 63) / 64, 64, 0, st>>>(cams0, xi, V, cams_out);
  return cudaGetLastError();
}

cudaError_t launch_adam_pose(float* xi, float* grad, float* m, float* s, int32_t* step, int V,
                             const gs_adam_config& hp, const float* loss, float* best_loss, float* best_xi,
                             cudaStream_t st) {
  k_adam_pose<<<1, 1024, 0, st>>>(xi, grad, m, s, step, V, hp, loss, best_loss, best_xi);
  return cudaGetLastError();
}

}  // namespace gsb

namespace gsb {

// Sparse Adam over the map (Sec. "Additional Strategies" (a)): only the
// Gaussians that take part in the rendering of the last projected batch (the
// workspace's list of Gaussians seen by some view) are updated; the others
// keep their parameters and moments.  One thread per listed Gaussian walks its
// parameter rows; the gradients of the updated Gaussians are cleared, so the
// gradient buffers are zero again for the next backward pass without a clear
// of the whole map.
__global__ void __launch_bounds__(256) k_sparse_adam(Ws ws, int32_t K, gs_param_set p, gs_param_set g,
                                                     gs_param_set m, gs_param_set v, const int32_t* __restrict__ step,
                                                     gs_adam_map_config hp) {
  const uint32_t count = ws.counters[kGaussCount];
  const int64_t n = ws.n;
  const float t = (float)(*step + 1);
  const float c1 = 1.f / (1.f - powf(hp.beta1, t)), c2 = 1.f / (1.f - powf(hp.beta2, t));
  for (uint64_t li = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; li < count;
       li += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t gi = ws.gauss_list[li];
    auto rows = [&](float* P, float* G, float* M, float* S, int nrows, float lr) {
      for (int r = 0; r < nrows; ++r) {
        const int64_t e = (int64_t)r * n + gi;
        const float gr = G[e];
        const float mi = hp.beta1 * M[e] + (1.f - hp.beta1) * gr;
        const float si = hp.beta2 * S[e] + (1.f - hp.beta2) * gr * gr;
        M[e] = mi;
        S[e] = si;
        P[e] -= lr * (mi * c1) / (sqrtf(si * c2) + hp.eps);
        G[e] = 0.f;
      }
    };
    rows(p.mean, g.mean, m.mean, v.mean, 3, hp.lr_mean);
    rows(p.log_scale, g.log_scale, m.log_scale, v.log_scale, 3, hp.lr_log_scale);
    rows(p.quat, g.quat, m.quat, v.quat, 4, hp.lr_quat);
    rows(p.logit_opacity, g.logit_opacity, m.logit_opacity, v.logit_opacity, 1, hp.lr_logit_opacity);
    rows(p.sh_dc, g.sh_dc, m.sh_dc, v.sh_dc, 3, hp.lr_sh_dc);
    if (K > 1) rows(p.sh_rest, g.sh_rest, m.sh_rest, v.sh_rest, 3 * (K - 1), hp.lr_sh_rest);
  }
}

__global__ void k_step_advance(int32_t* step) { *step += 1; }

cudaError_t launch_sparse_adam(const Ws& ws, int32_t sh_degree, const gs_param_set& p, const gs_param_set& g,
                               const gs_param_set& m, const gs_param_set& v, int32_t* step,
                               const gs_adam_map_config& hp, cudaStream_t st) {
  const int32_t K = (sh_degree + 1) * (sh_degree + 1);
  const int64_t need = (ws.n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  trace_begin(kKSparseAdam, st);
  k_sparse_adam<<<(unsigned)(need < cap ? need : cap), 256, 0, st>>>(ws, K, p, g, m, v, step, hp);
  trace_end(st);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_step_advance<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

}  // namespace gsb
