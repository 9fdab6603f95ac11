// C ABI of the rasterizer: argument checks, workspace layout, launches.
// The operations themselves are defined in the header next to each entry
// point (arxiv 2507.04004 references there).
#include <cmath>
#include <cstring>

#include "gs_internal.h"

namespace gsb {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static bool frame_ok(const gs_frame* f) {
  return f && f->n_views >= 1 && f->n_views <= 65535 && f->width >= 1 && f->width <= 8192 && f->height >= 1 &&
         f->height <= 8192;
}

static gs_status layout(int64_t n, const gs_frame* f, int64_t cap, gs_layout* L) {
  if (!L || !frame_ok(f) || n < 1 || n >= (int64_t(1) << 31) || cap < 1 || cap >= (int64_t(1) << 31))
    return GS_ERR_ARG;
  const int64_t V = f->n_views;
  const int64_t E = V * n;
  if (E >= (int64_t(1) << 30)) return GS_ERR_UNSUPPORTED;  // the sort's status words hold 30-bit counts
  const int64_t T = (int64_t)((f->width + 15) / 16) * ((f->height + 15) / 16);
  if (V * T >= (int64_t(1) << 31)) return GS_ERR_UNSUPPORTED;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  const int64_t tx = (f->width + 15) / 16, ty = (f->height + 15) / 16;
  const int64_t B = V * ty;
  const int64_t units_e = (E + kEntryUnit - 1) / kEntryUnit + V * (unit_ramp(kEntryUnit) + 1);
  const int64_t units_r = (cap + kRowUnit - 1) / kRowUnit + B * (unit_ramp(kRowUnit) + 1);
  L->counters = take(16 * sizeof(uint32_t));
  L->records = take((size_t)E * 3 * sizeof(float4));
  L->rects = take((size_t)E * sizeof(uint2));
  L->adjoints = take((size_t)E * 3 * sizeof(float4));
  L->visible = take((size_t)E * sizeof(uint32_t));
  L->vis_key = take((size_t)E * sizeof(uint32_t));
  L->sort_key = take((size_t)2 * E * sizeof(uint32_t));
  L->sort_val = take((size_t)2 * E * sizeof(uint32_t));
  L->radix_status = take((size_t)6 * 256 * (1 + (E + kRadixTileEntries - 1) / kRadixTileEntries) * sizeof(uint32_t));
  L->view_start = take((size_t)(V + 1) * sizeof(uint32_t));
  L->gauss_list = take((size_t)n * sizeof(uint32_t));
  L->tile_count = take((size_t)(V * T) * sizeof(uint32_t));
  L->tile_start = take((size_t)(V * T) * sizeof(uint32_t));
  L->bucket_count = take((size_t)B * sizeof(uint32_t));
  L->bucket_start = take((size_t)B * sizeof(uint32_t));
  L->unit_first_e = take((size_t)(V + 1) * sizeof(uint32_t));
  L->unit_seg_e = take((size_t)units_e * sizeof(uint32_t));
  L->unit_cnt_e = take((size_t)units_e * ty * sizeof(uint32_t));
  L->unit_first_r = take((size_t)(B + 1) * sizeof(uint32_t));
  L->unit_seg_r = take((size_t)units_r * sizeof(uint32_t));
  L->unit_cnt_r = take((size_t)units_r * tx * sizeof(uint32_t));
  L->row_items = take((size_t)cap * sizeof(uint32_t));
  L->row_span = take((size_t)cap * sizeof(uint32_t));
  L->sorted_ids = take((size_t)cap * sizeof(uint32_t));
  // view_stats and work_fill stay adjacent: the blend backward clears both with one memset
  L->view_stats = take((size_t)V * 4 * sizeof(float));
  L->work_fill = take((size_t)kWorkClasses * sizeof(uint32_t));
  L->work_lists = take((size_t)kWorkClasses * (V * T) * sizeof(uint32_t));
  L->total = off;
  return GS_OK;
}

Ws resolve_ws(const gs_workspace* w, const gs_layout& L) {
  char* b = static_cast<char*>(w->ptr);
  auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t*>(b + off); };
  Ws ws;
  ws.counters = u32(L.counters);
  ws.records = reinterpret_cast<float4*>(b + L.records);
  ws.rects = reinterpret_cast<uint2*>(b + L.rects);
  ws.adjoints = reinterpret_cast<float4*>(b + L.adjoints);
  ws.visible = u32(L.visible);
  ws.vis_key = u32(L.vis_key);
  ws.sort_key = u32(L.sort_key);
  ws.sort_val = u32(L.sort_val);
  // the sort's last pass writes the entry buffer (passes - 1) & 1, which
  // k_entry_order reads: the other one holds the sorted list from then on
  ws.sorted = ws.sort_val + (size_t)(depth_sort_passes(w->frame.n_views) & 1) * (size_t)w->frame.n_views * (size_t)w->n;
  ws.radix_status = u32(L.radix_status);
  ws.view_start = u32(L.view_start);
  ws.gauss_list = u32(L.gauss_list);
  ws.tile_count = u32(L.tile_count);
  ws.tile_start = u32(L.tile_start);
  ws.bucket_count = u32(L.bucket_count);
  ws.bucket_start = u32(L.bucket_start);
  ws.unit_first_e = u32(L.unit_first_e);
  ws.unit_seg_e = u32(L.unit_seg_e);
  ws.unit_cnt_e = u32(L.unit_cnt_e);
  ws.unit_first_r = u32(L.unit_first_r);
  ws.unit_seg_r = u32(L.unit_seg_r);
  ws.unit_cnt_r = u32(L.unit_cnt_r);
  ws.row_items = u32(L.row_items);
  ws.row_span = u32(L.row_span);
  ws.sorted_ids = u32(L.sorted_ids);
  ws.view_stats = reinterpret_cast<float*>(b + L.view_stats);
  ws.work_fill = u32(L.work_fill);
  ws.work_lists = u32(L.work_lists);
  ws.n = w->n;
  ws.cap = w->pair_capacity;
  ws.views = w->frame.n_views;
  ws.width = w->frame.width;
  ws.height = w->frame.height;
  ws.tiles_x = (ws.width + 15) / 16;
  ws.tiles_y = (ws.height + 15) / 16;
  ws.tiles_per_view = ws.tiles_x * ws.tiles_y;
  ws.units_e_max = ((int64_t)ws.views * ws.n + kEntryUnit - 1) / kEntryUnit + ws.views * (unit_ramp(kEntryUnit) + 1);
  ws.units_r_max = (ws.cap + kRowUnit - 1) / kRowUnit + (int64_t)ws.views * ws.tiles_y * (unit_ramp(kRowUnit) + 1);
  ws.radix_tiles_max = ((int64_t)ws.views * ws.n + kRadixTileEntries - 1) / kRadixTileEntries;
  return ws;
}

int sm_count() {
  int dev = 0, n = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

static gs_status check_ws(const gs_workspace* w, gs_layout* L) {
  if (!w || !w->ptr) return GS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(w->ptr) & 255u) != 0) return GS_ERR_ARG;
  return layout(w->n, &w->frame, w->pair_capacity, L);
}

static gs_status check_map(const gs_map* m, const gs_workspace* w) {
  if (!m || m->n != w->n || m->sh_degree < 0 || m->sh_degree > 3 || (m->sh_bf16 != 0 && m->sh_bf16 != 1))
    return GS_ERR_ARG;
  if (!m->mean || !m->log_scale || !m->quat || !m->logit_opacity || !m->sh_dc) return GS_ERR_ARG;
  if (m->sh_degree > 0 && !m->sh_rest) return GS_ERR_ARG;
  return GS_OK;
}

static gs_status check_cfg(const gs_config* c) {
  if (!c) return GS_ERR_ARG;
  if (!(c->alpha_min > 0.f && c->alpha_min < 1.f) || !(c->alpha_max >= c->alpha_min && c->alpha_max < 1.f) ||
      !(c->t_min > 0.f && c->t_min < 1.f) || !(c->near_z > 0.f) || !(c->dilation >= 0.f) || !(c->fov_clamp > 0.f))
    return GS_ERR_ARG;
  return GS_OK;
}

static gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

// Tracing state (single host thread drives the library while tracing).
static struct {
  cudaEvent_t* events = nullptr;
  int32_t* ids = nullptr;
  int32_t capacity = 0;
  int32_t count = 0;
  bool on = false;
} g_trace;

void trace_begin(int kernel_id, cudaStream_t st) {
  if (!g_trace.on) return;
  const int k = g_trace.count;
  if (k < g_trace.capacity) {
    cudaEventRecord(g_trace.events[2 * k], st);
    if (g_trace.ids) g_trace.ids[k] = kernel_id;
  }
}

void trace_end(cudaStream_t st) {
  if (!g_trace.on) return;
  const int k = g_trace.count++;
  if (k < g_trace.capacity) cudaEventRecord(g_trace.events[2 * k + 1], st);
}

}  // namespace gsb

using namespace gsb;

extern "C" {

size_t gs_workspace_size(int64_t n, const gs_frame* frame, int64_t pair_capacity) {
  gs_layout L;
  return layout(n, frame, pair_capacity, &L) == GS_OK ? L.total : 0;
}

gs_status gs_workspace_layout(int64_t n, const gs_frame* frame, int64_t pair_capacity, gs_layout* out) {
  return layout(n, frame, pair_capacity, out);
}

gs_status gs_read_status(const gs_workspace* ws, gs_stream_t stream, int32_t* status_out, int64_t* pairs_needed_out) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  uint32_t c[2] = {0, 0};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(c, static_cast<char*>(ws->ptr) + L.counters, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (status_out) *status_out = (int32_t)c[0];
  if (pairs_needed_out) *pairs_needed_out = (int64_t)c[1];
  return GS_OK;
}

gs_status gs_project(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg, const gs_workspace* ws,
                     gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if ((s = check_map(map, ws)) != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!cams_dev) return GS_ERR_ARG;
  const Ws w = resolve_ws(ws, L);
  return cuda_status(launch_project(*map, cams_dev, *cfg, w, reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_bin_sort(const gs_workspace* ws, gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  return cuda_status(launch_bin_sort(resolve_ws(ws, L), reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_render_fwd(const gs_config* cfg, const gs_workspace* ws, float* rgb, float* depth, float* opac,
                        float* t_final, uint32_t* n_contrib, gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!t_final || !n_contrib) return GS_ERR_ARG;
  return cuda_status(launch_render_fwd(*cfg, resolve_ws(ws, L), rgb, depth, opac, t_final, n_contrib,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_blend_counts(const gs_config* cfg, const gs_workspace* ws, uint64_t* counts_dev, gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!counts_dev || (reinterpret_cast<uintptr_t>(counts_dev) & 7u) != 0) return GS_ERR_ARG;
  return cuda_status(launch_blend_counts(*cfg, resolve_ws(ws, L), reinterpret_cast<unsigned long long*>(counts_dev),
                                         reinterpret_cast<cudaStream_t>(stream)));
}

// Argument checks and marshalling shared by both blend backwards.
static gs_status bwd_args(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg, const gs_workspace* ws,
                          const float* rgb, const float* depth, const float* opac, const float* t_final,
                          const uint32_t* n_contrib, const float* tgt_rgb, const float* tgt_depth, float w_rgb,
                          float w_depth, const float* dl_drgb, const float* dl_ddepth, const float* dl_dopac,
                          float* grad_mean, float* grad_log_scale, float* grad_quat, float* grad_logit_opacity,
                          float* grad_sh_dc, float* grad_sh_rest, float* grad_pose, float* loss_out, gs_layout* L,
                          BwdArgs* out, const uint8_t* tgt_rgb8 = nullptr) {
  gs_status s = check_ws(ws, L);
  if (s != GS_OK) return s;
  if ((s = check_map(map, ws)) != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!cams_dev || !t_final || !n_contrib) return GS_ERR_ARG;
  // parameter gradients: all given, or none (pose gradient only)
  const bool params = grad_mean || grad_log_scale || grad_quat || grad_logit_opacity || grad_sh_dc || grad_sh_rest;
  if (params) {
    if (!grad_mean || !grad_log_scale || !grad_quat || !grad_logit_opacity || !grad_sh_dc) return GS_ERR_ARG;
    if (map->sh_degree > 0 && !grad_sh_rest) return GS_ERR_ARG;
  } else if (!grad_pose) {
    return GS_ERR_ARG;
  }
  if (tgt_rgb && tgt_rgb8) return GS_ERR_ARG;
  if (tgt_rgb || tgt_rgb8) {
    if (!rgb) return GS_ERR_ARG;
    if (tgt_depth && w_depth != 0.f && (!depth || !opac)) return GS_ERR_ARG;
  }
  BwdArgs a;
  a.rgb = rgb; a.depth = depth; a.opac = opac; a.t_final = t_final; a.n_contrib = n_contrib;
  a.tgt_rgb = tgt_rgb; a.tgt_rgb8 = tgt_rgb8; a.tgt_depth = tgt_depth; a.w_rgb = w_rgb; a.w_depth = w_depth;
  a.dl_drgb = dl_drgb; a.dl_ddepth = dl_ddepth; a.dl_dopac = dl_dopac;
  a.grad_mean = grad_mean; a.grad_log_scale = grad_log_scale; a.grad_quat = grad_quat;
  a.grad_logit = grad_logit_opacity; a.grad_sh_dc = grad_sh_dc; a.grad_sh_rest = grad_sh_rest;
  a.grad_pose = grad_pose; a.loss = loss_out;
  *out = a;
  return GS_OK;
}

gs_status gs_render_bwd(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg, const gs_workspace* ws,
                        const float* rgb, const float* depth, const float* opac, const float* t_final,
                        const uint32_t* n_contrib, const float* tgt_rgb, const float* tgt_depth, float w_rgb,
                        float w_depth, const float* dl_drgb, const float* dl_ddepth, const float* dl_dopac,
                        float* grad_mean, float* grad_log_scale, float* grad_quat, float* grad_logit_opacity,
                        float* grad_sh_dc, float* grad_sh_rest, float* grad_pose, float* loss_out,
                        gs_stream_t stream) {
  gs_layout L;
  BwdArgs a;
  const gs_status s = bwd_args(map, cams_dev, cfg, ws, rgb, depth, opac, t_final, n_contrib, tgt_rgb, tgt_depth,
                               w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale, grad_quat,
                               grad_logit_opacity, grad_sh_dc, grad_sh_rest, grad_pose, loss_out, &L, &a);
  if (s != GS_OK) return s;
  return cuda_status(launch_render_bwd(*map, cams_dev, *cfg, resolve_ws(ws, L), a,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_render_bwd_rgb8(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                             const gs_workspace* ws, const float* rgb, const float* depth, const float* opac,
                             const float* t_final, const uint32_t* n_contrib, const uint8_t* tgt_rgb8,
                             const float* tgt_depth, float w_rgb, float w_depth, const float* dl_drgb,
                             const float* dl_ddepth, const float* dl_dopac, float* grad_mean, float* grad_log_scale,
                             float* grad_quat, float* grad_logit_opacity, float* grad_sh_dc, float* grad_sh_rest,
                             float* grad_pose, float* loss_out, gs_stream_t stream) {
  if (!tgt_rgb8) return GS_ERR_ARG;
  gs_layout L;
  BwdArgs a;
  const gs_status s = bwd_args(map, cams_dev, cfg, ws, rgb, depth, opac, t_final, n_contrib, nullptr, tgt_depth,
                               w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale, grad_quat,
                               grad_logit_opacity, grad_sh_dc, grad_sh_rest, grad_pose, loss_out, &L, &a, tgt_rgb8);
  if (s != GS_OK) return s;
  return cuda_status(launch_render_bwd(*map, cams_dev, *cfg, resolve_ws(ws, L), a,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

size_t gs_bucket_workspace_size(const gs_workspace* ws) {
  gs_layout L;
  if (check_ws(ws, &L) != GS_OK) return 0;
  return bucket_ws_bytes(resolve_ws(ws, L));
}

gs_status gs_render_fwd_checkpointed(const gs_config* cfg, const gs_workspace* ws, float* rgb, float* depth,
                                     float* opac, float* t_final, uint32_t* n_contrib, void* bucket_ws,
                                     gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!t_final || !n_contrib || !bucket_ws || (reinterpret_cast<uintptr_t>(bucket_ws) & 255u)) return GS_ERR_ARG;
  const Ws w = resolve_ws(ws, L);
  return cuda_status(launch_render_fwd_ckpt(*cfg, w, rgb, depth, opac, t_final, n_contrib,
                                            resolve_bucket_ws(w, bucket_ws).ckpt,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_render_bwd_buckets(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                                const gs_workspace* ws, const float* rgb, const float* depth, const float* opac,
                                const float* t_final, const uint32_t* n_contrib, const float* tgt_rgb,
                                const float* tgt_depth, float w_rgb, float w_depth, const float* dl_drgb,
                                const float* dl_ddepth, const float* dl_dopac, float* grad_mean,
                                float* grad_log_scale, float* grad_quat, float* grad_logit_opacity,
                                float* grad_sh_dc, float* grad_sh_rest, float* grad_pose, float* loss_out,
                                const void* bucket_ws, gs_stream_t stream) {
  gs_layout L;
  BwdArgs a;
  const gs_status s = bwd_args(map, cams_dev, cfg, ws, rgb, depth, opac, t_final, n_contrib, tgt_rgb, tgt_depth,
                               w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale, grad_quat,
                               grad_logit_opacity, grad_sh_dc, grad_sh_rest, grad_pose, loss_out, &L, &a);
  if (s != GS_OK) return s;
  if (!rgb || !depth || !bucket_ws || (reinterpret_cast<uintptr_t>(bucket_ws) & 255u)) return GS_ERR_ARG;
  const Ws w = resolve_ws(ws, L);
  return cuda_status(launch_render_bwd_bucket(*map, cams_dev, *cfg, w, a,
                                              resolve_bucket_ws(w, const_cast<void*>(bucket_ws)),
                                              reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_pose_jacobian(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                           const gs_workspace* ws, const int32_t* pix_idx, int32_t n_pix, float* J, float* rgb_out,
                           gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if ((s = check_map(map, ws)) != GS_OK) return s;
  if ((s = check_cfg(cfg)) != GS_OK) return s;
  if (!cams_dev || !pix_idx || !J || n_pix < 1) return GS_ERR_ARG;
  return cuda_status(launch_pose_jacobian(*map, cams_dev, *cfg, resolve_ws(ws, L), pix_idx, n_pix, J, rgb_out,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_sparse_adam(const gs_workspace* ws, int32_t sh_degree, const gs_param_set* params,
                         const gs_param_set* grads, const gs_param_set* m, const gs_param_set* v, int32_t* step_dev,
                         const gs_adam_map_config* cfg, gs_stream_t stream) {
  gs_layout L;
  gs_status s = check_ws(ws, &L);
  if (s != GS_OK) return s;
  if (!params || !grads || !m || !v || !step_dev || !cfg || sh_degree < 0 || sh_degree > 3) return GS_ERR_ARG;
  for (const gs_param_set* q : {params, grads, m, v}) {
    if (!q->mean || !q->log_scale || !q->quat || !q->logit_opacity || !q->sh_dc) return GS_ERR_ARG;
    if (sh_degree > 0 && !q->sh_rest) return GS_ERR_ARG;
  }
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps > 0.f))
    return GS_ERR_ARG;
  return cuda_status(launch_sparse_adam(resolve_ws(ws, L), sh_degree, *params, *grads, *m, *v, step_dev, *cfg,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_unpack_keyframes(const uint8_t* rgb8_dev, int32_t n_views, int32_t height, int32_t width,
                              float* rgb_dev, const int32_t* depth_idx_dev, const float* depth_val_dev,
                              const int32_t* depth_offsets_dev, float* depth_dev, gs_stream_t stream) {
  if (!rgb8_dev != !rgb_dev || n_views < 1 || height < 1 || width < 1) return GS_ERR_ARG;
  if (!rgb8_dev && !depth_dev) return GS_ERR_ARG;  // nothing to unpack
  if (depth_idx_dev && (!depth_val_dev || !depth_offsets_dev || !depth_dev)) return GS_ERR_ARG;
  return cuda_status(launch_unpack_keyframes(rgb8_dev, n_views, height, width, rgb_dev, depth_idx_dev, depth_val_dev,
                                             depth_offsets_dev, depth_dev, reinterpret_cast<cudaStream_t>(stream)));
}

size_t gs_expand_scratch_bytes(int64_t n_points) {
  if (n_points < 1 || n_points >= (int64_t(1) << 31)) return 0;
  return expand_scratch_bytes(n_points);
}

gs_status gs_expand_select(const float* points_dev, int64_t n_points, const gs_camera* cam_dev, const gs_config* cfg,
                           const float* opac_dev, int32_t height, int32_t width, float tau, void* scratch,
                           int32_t* idx_out, uint32_t* count_out, gs_stream_t stream) {
  if (!points_dev || !cam_dev || !opac_dev || !scratch || !idx_out || !count_out) return GS_ERR_ARG;
  if (n_points < 1 || n_points >= (int64_t(1) << 31) || height < 1 || width < 1) return GS_ERR_ARG;
  gs_status s = check_cfg(cfg);
  if (s != GS_OK) return s;
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return GS_ERR_ARG;
  return cuda_status(launch_expand_select(points_dev, n_points, cam_dev, opac_dev, height, width, tau, cfg->near_z,
                                          scratch, idx_out, count_out, reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_expand_init(const float* points_dev, const float* rgb_dev, int64_t n_points, const int32_t* idx_dev,
                         const uint32_t* count_dev, const gs_camera* cam_dev, int64_t first, const gs_param_set* dst,
                         int64_t n_dst, int32_t sh_degree, float init_opacity, gs_stream_t stream) {
  if (!points_dev || !rgb_dev || !idx_dev || !count_dev || !cam_dev || !dst) return GS_ERR_ARG;
  if (n_points < 1 || first < 0 || n_dst < first || sh_degree < 0 || sh_degree > 3) return GS_ERR_ARG;
  if (!dst->mean || !dst->log_scale || !dst->quat || !dst->logit_opacity || !dst->sh_dc) return GS_ERR_ARG;
  if (sh_degree > 0 && !dst->sh_rest) return GS_ERR_ARG;
  if (!(init_opacity > 0.f && init_opacity < 1.f)) return GS_ERR_ARG;
  const float logit = std::log(init_opacity / (1.f - init_opacity));
  return cuda_status(launch_expand_init(points_dev, rgb_dev, n_points, idx_dev, count_dev, cam_dev, first, n_dst,
                                        sh_degree, logit, *dst, reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_pose_apply(const gs_camera* cams0_dev, const float* xi_dev, int32_t n_views, gs_camera* cams_out_dev,
                        gs_stream_t stream) {
  if (!cams0_dev || !xi_dev || !cams_out_dev || n_views < 1) return GS_ERR_ARG;
  return cuda_status(launch_pose_apply(cams0_dev, xi_dev, n_views, cams_out_dev,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_pose_residual(const gs_camera* cams_traj_dev, const gs_camera* cams_opt_dev, int32_t n_views,
                           float* r_dev, gs_stream_t stream) {
  if (!cams_traj_dev || !cams_opt_dev || !r_dev || n_views < 1) return GS_ERR_ARG;
  return cuda_status(launch_pose_residual(cams_traj_dev, cams_opt_dev, n_views, r_dev,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_adam_pose(float* xi_dev, float* grad_dev, float* m_dev, float* v_dev, int32_t* step_dev,
                       int32_t n_views, const gs_adam_config* cfg, const float* loss_dev, float* best_loss_dev,
                       float* best_xi_dev, gs_stream_t stream) {
  if (!xi_dev || !grad_dev || !m_dev || !v_dev || !step_dev || !cfg || n_views < 1) return GS_ERR_ARG;
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps > 0.f))
    return GS_ERR_ARG;
  if ((loss_dev || best_loss_dev || best_xi_dev) && !(loss_dev && best_loss_dev && best_xi_dev)) return GS_ERR_ARG;
  return cuda_status(launch_adam_pose(xi_dev, grad_dev, m_dev, v_dev, step_dev, n_views, *cfg, loss_dev,
                                      best_loss_dev, best_xi_dev, reinterpret_cast<cudaStream_t>(stream)));
}

size_t gs_dssim_scratch_bytes(int32_t n_views, int32_t height, int32_t width) {
  if (n_views < 1 || height < 1 || width < 1) return 0;
  return dssim_scratch_bytes(n_views, height, width);
}

gs_status gs_dssim(const float* img, const float* tgt, int32_t n_views, int32_t height, int32_t width, float weight,
                   float* loss, float* dl_dimg, void* scratch, gs_stream_t stream) {
  if (!img || !tgt || !scratch || n_views < 1 || height < 1 || width < 1) return GS_ERR_ARG;
  if ((int64_t)n_views * 3 > 65535) return GS_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return GS_ERR_ARG;
  return cuda_status(launch_dssim(img, tgt, n_views, height, width, weight, loss, dl_dimg, scratch,
                                  reinterpret_cast<cudaStream_t>(stream)));
}

gs_status gs_trace_start(void* const* events, int32_t capacity, int32_t* kernel_ids) {
  if (!events || capacity < 1) return GS_ERR_ARG;
  g_trace.events = reinterpret_cast<cudaEvent_t*>(const_cast<void**>(events));
  g_trace.ids = kernel_ids;
  g_trace.capacity = capacity;
  g_trace.count = 0;
  g_trace.on = true;
  return GS_OK;
}

int32_t gs_trace_stop(void) {
  g_trace.on = false;
  return g_trace.count;
}

const char* gs_kernel_name(int32_t id) {
  static const char* names[kKNumKernels] = {
      "project",    "scan",           "scatter_rows",   "depth_hist",    "depth_scan",  "render_fwd",
      "count_depth", "render_bwd",    "preprocess_bwd", "pose_jacobian", "scan_buckets", "rows_count",
      "rows_emit",  "ssim_fwd",       "ssim_bwd",       "sparse_adam",   "depth_scatter", "render_fwd_ckpt",
      "render_bwd_bucket", "entry_order", "entry_units", "entry_rows",   "unit_scan", "tile_work"};
  return (id >= 0 && id < kKNumKernels) ? names[id] : "unknown";
}

const char* gs_status_str(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "pair buffer too small";
    case GS_ERR_OOM: return "out of memory";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_TIMEOUT: return "device wait timed out";
    case GS_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char* gs_version(void) { return "gsb300 0.1"; }

}  // extern "C"
