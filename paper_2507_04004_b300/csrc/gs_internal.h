// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "gs.h"
#include "gs_device.cuh"

namespace gsb {

// Kernel ids reported by the tracing hook (gs_trace_start).
enum KernelId {
  kKProject = 0, kKScan, kKScatterRows, kKDepthHist, kKDepthScan, kKRenderFwd, kKCountDepth, kKRenderBwd,
  kKPreprocessBwd, kKPoseJacobian, kKScanBuckets, kKRowsCount, kKRowsEmit, kKSsimFwd, kKSsimBwd, kKSparseAdam,
  kKDepthScatter, kKRenderFwdCkpt, kKRenderBwdBucket, kKEntryOrder, kKEntryUnits, kKEntryRows, kKUnitScan,
  kKTileWork, kKNumKernels
};
// Bracket one kernel launch with the caller's trace events (no-op when off).
void trace_begin(int kernel_id, cudaStream_t st);
void trace_end(cudaStream_t st);

// Resolve the device view of a caller workspace (layout must be valid).
Ws resolve_ws(const gs_workspace* ws, const gs_layout& L);
int sm_count();

cudaError_t launch_project(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                           cudaStream_t st);
cudaError_t launch_bin_sort(const Ws& ws, cudaStream_t st);
size_t dssim_scratch_bytes(int V, int H, int W);
cudaError_t launch_sparse_adam(const Ws& ws, int32_t sh_degree, const gs_param_set& p, const gs_param_set& g,
                               const gs_param_set& m, const gs_param_set& v, int32_t* step,
                               const gs_adam_map_config& hp, cudaStream_t st);
cudaError_t launch_unpack_keyframes(const uint8_t* rgb8, int V, int H, int W, float* rgb, const int32_t* idx,
                                    const float* val, const int32_t* offsets, float* depth, cudaStream_t st);
size_t expand_scratch_bytes(int64_t P);
cudaError_t launch_expand_select(const float* pts, int64_t P, const gs_camera* cam, const float* opac, int H, int W,
                                 float tau, float near, void* scratch, int32_t* out_idx, uint32_t* count,
                                 cudaStream_t st);
cudaError_t launch_expand_init(const float* pts, const float* rgb, int64_t P, const int32_t* idx,
                               const uint32_t* count, const gs_camera* cam, int64_t first, int64_t n_dst,
                               int32_t sh_degree, float logit_init, const gs_param_set& dst, cudaStream_t st);
cudaError_t launch_pose_apply(const gs_camera* cams0, const float* xi, int V, gs_camera* cams_out, cudaStream_t st);
cudaError_t launch_pose_residual(const gs_camera* cams_a, const gs_camera* cams_b, int V, float* r, cudaStream_t st);
cudaError_t launch_adam_pose(float* xi, float* grad, float* m, float* s, int32_t* step, int V,
                             const gs_adam_config& hp, const float* loss, float* best_loss, float* best_xi,
                             cudaStream_t st);
cudaError_t launch_dssim(const float* img, const float* tgt, int V, int H, int W, float weight, float* loss,
                         float* dl_dimg, void* scratch, cudaStream_t st);
cudaError_t launch_render_fwd(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                              float* t_final, uint32_t* n_contrib, cudaStream_t st);
cudaError_t launch_blend_counts(const gs_config& cfg, const Ws& ws, unsigned long long* counts, cudaStream_t st);

struct BwdArgs {
  const float *rgb, *depth, *opac, *t_final;
  const uint32_t* n_contrib;
  const float *tgt_rgb, *tgt_depth;
  const uint8_t* tgt_rgb8;  // 8-bit colour targets (c / 255) in place of tgt_rgb, or null
  bool fused() const { return tgt_rgb != nullptr || tgt_rgb8 != nullptr; }
  float w_rgb, w_depth;
  const float *dl_drgb, *dl_ddepth, *dl_dopac;
  float *grad_mean, *grad_log_scale, *grad_quat, *grad_logit, *grad_sh_dc, *grad_sh_rest, *grad_pose, *loss;
};
cudaError_t launch_render_bwd(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                              const BwdArgs& a, cudaStream_t st);
// Stages shared by both blend backwards: per-view loss accumulators and
// valid-depth counts before the blend stage, the projection backward after it.
cudaError_t launch_bwd_prologue(const Ws& ws, const BwdArgs& a, cudaStream_t st);
cudaError_t launch_preprocess_bwd(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                  const BwdArgs& a, cudaStream_t st);
// Per-Gaussian (bucket) backward: the checkpoints written by the forward, in
// one caller buffer of bucket_ws_bytes(ws) bytes.
struct BucketWs {
  float* ckpt;   // [cap / 32 + V*T + 1][5][256]: T, C_r, C_g, C_b, D at each bucket start
};
size_t bucket_ws_bytes(const Ws& ws);
BucketWs resolve_bucket_ws(const Ws& ws, void* ptr);
cudaError_t launch_render_fwd_ckpt(const gs_config& cfg, const Ws& ws, float* rgb, float* depth, float* opac,
                                   float* t_final, uint32_t* n_contrib, float* ckpt, cudaStream_t st);
cudaError_t launch_render_bwd_bucket(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                     const BwdArgs& a, const BucketWs& bw, cudaStream_t st);
cudaError_t launch_pose_jacobian(const gs_map& map, const gs_camera* cams, const gs_config& cfg, const Ws& ws,
                                 const int32_t* pix, int32_t n_pix, float* J, float* rgb, cudaStream_t st);

}  // namespace gsb
