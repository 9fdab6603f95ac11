/*
 * gs.h - C ABI of the B300 (sm_103a) differentiable tile-based 3D Gaussian
 * splatting rasterizer of Gaussian-LIC2 (arxiv 2507.04004).
 *
 * The library renders RGB, depth and opacity of a Gaussian map at a batch of
 * camera poses (Sec. "3D Gaussian Splatting Representation": projection,
 * Eq. alpha, Eq. rendered_rgb, Eq. rendered_depth, Eq. rendered_opacity), with
 * the tile culling of Sec. "Fast Tile-based Culling", and back-propagates the
 * depth-regularised loss of Eq. depth_loss (L1 colour term plus the
 * opacity-normalised sparse LiDAR depth term) to the Gaussian parameters and to
 * the camera pose (Eq. 3dgs_jacobi under the right perturbation T Exp(xi)).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev, and every array argument unless stated otherwise,
 *     are device pointers owned by the caller; the library never allocates,
 *     frees or retains them beyond the call.  gs_map, gs_frame, gs_config and
 *     gs_workspace are host structs passed by pointer and read during the call.
 *   - Every call is asynchronous on the given CUDA stream (NULL = legacy
 *     default stream) and only enqueues work; argument errors are returned
 *     synchronously and enqueue nothing.  Conditions found on the device
 *     (pair-buffer overflow) are written to the workspace status word, read
 *     with gs_read_status() after the stream has been synchronised.
 *   - Nothing is thrown across the ABI and no device code traps or asserts.
 *   - Images are planar: rgb is [V][3][H][W], depth/opacity/t_final/n_contrib
 *     are [V][H][W], row-major, pixel (i, j) sampled at (i + 0.5, j + 0.5).
 *   - Gaussian parameters are structure-of-arrays, channel-major: mean [3][N],
 *     log_scale [3][N], quat [4][N] as (w, x, y, z) (normalised inside),
 *     logit_opacity [N], sh_dc [3][N], sh_rest [K-1][3][N] with
 *     K = (sh_degree + 1)^2 and the real SH basis (Condon-Shortley phase,
 *     m = -l..l inside each degree).  SH arrays are FP32, or BF16 when
 *     sh_bf16 != 0; all arithmetic is FP32.
 *   - A camera is the world-to-camera transform (row-major R, t) and pinhole
 *     intrinsics.  All views of one call share width and height.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream_t; /* same type as cudaStream_t */

typedef enum {
  GS_OK = 0,
  GS_ERR_ARG = 1,         /* invalid argument (null pointer, size, degree, ...) */
  GS_ERR_CAPACITY = 2,    /* (device status) pair buffer too small; see gs_read_status */
  GS_ERR_OOM = 3,         /* reserved for callers' allocators; never returned by the library */
  GS_ERR_CUDA = 4,        /* a CUDA launch or runtime call failed */
  GS_ERR_TIMEOUT = 5,     /* (device status) a bounded device wait gave up */
  GS_ERR_UNSUPPORTED = 6  /* valid request outside the supported envelope */
} gs_status;

/* One camera; an array of these lives in device memory (64 bytes each). */
typedef struct {
  float R[9]; /* world-to-camera rotation, row-major */
  float t[3]; /* world-to-camera translation */
  float fx, fy, cx, cy;
} gs_camera;

/* Gaussian map: host struct holding caller-owned device pointers. */
typedef struct {
  int64_t n;              /* number of Gaussians, >= 1, < 2^31 */
  int32_t sh_degree;      /* 0..3 */
  int32_t sh_bf16;        /* 0: SH arrays are float, 1: __nv_bfloat16 */
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* logit_opacity;
  const void* sh_dc;
  const void* sh_rest;    /* may be NULL when sh_degree == 0 */
} gs_map;

/* Batch geometry: n_views images of width x height (1..8192 each). */
typedef struct {
  int32_t n_views, width, height;
} gs_frame;

/* Rasterization constants (readings of the 3DGS rasterizer the paper builds
 * on): defaults 1/255, 0.99, 1e-4, 0.2, 0.3, 1.3, black background. */
typedef struct {
  float alpha_min;  /* skip a Gaussian at a pixel below this alpha; tile culling threshold */
  float alpha_max;  /* clamp of alpha */
  float t_min;      /* stop before a Gaussian that would take transmittance below this */
  float near_z;     /* cut Gaussians whose depth key is <= near_z */
  float dilation;   /* added to the diagonal of the 2D covariance, px^2 */
  float fov_clamp;  /* x/z, y/z clamp inside the affine Jacobian, in half fields of view */
  float bg[3];      /* background colour blended with the final transmittance */
} gs_config;

/* Workspace: one caller-allocated device buffer of gs_workspace_size() bytes
 * (256-byte aligned) holding projected Gaussians, tile bins, sort keys, 2D
 * adjoints and the device status word of one batch geometry.  It is written by
 * gs_project / gs_bin_sort and read by the later calls of the same batch. */
typedef struct {
  void* ptr;
  int64_t n;              /* Gaussians the workspace was sized for */
  int64_t pair_capacity;  /* (Gaussian, tile) pairs it can hold, < 2^31; also bounds the
                             (Gaussian, tile row) items of the binning pass */
  gs_frame frame;
} gs_workspace;

/* Byte offsets of the workspace's parts (for inspection and tests).  E = V*N
 * (view, Gaussian) entries, T tiles per view, B = V*ceil(H/16) (view, tile
 * row) buckets, cap the pair capacity; an entry unit is up to 256 sorted
 * visible entries of one view, a row unit up to 128 row items of one bucket. */
typedef struct {
  size_t counters;    /* uint32[16]: [0] status, [1] pairs (or row items) needed, [2] visible entries,
                         [3] entry units, [4] row items, [5] Gaussians in gauss_list, [6] row units,
                         [8..13] tile tickets of the sort's passes, [15] chunk tickets of the projection */
  size_t records;     /* float4[E][3]: (mx, my, conic a, conic b), (conic c, opacity, depth, -), (r, g, b, -) */
  size_t rects;       /* uint32[E][2]: tile box (x0 | y0 << 16, x1 | y1 << 16), empty when x0 > x1 */
  size_t adjoints;    /* float4[E][3]: 2D adjoints (mx, my, a, b), (c, o, depth, -), (r, g, b, -) */
  size_t visible;     /* uint32[E]: entries v*N + g with a non-empty box, after binning in
                         (view, depth key, Gaussian index) order */
  size_t vis_key;     /* uint32[E]: depth key bits of the visible entries (projection order) */
  size_t sort_key;    /* uint32[2][E]: radix-sort buffers (keys) */
  size_t sort_val;    /* uint32[2][E]: radix-sort buffers (entries) */
  size_t radix_status; /* uint32[6][256] digit counts of the sort's passes, then
                          uint32[6][ceil(E/2048)][256] per-tile status words */
  size_t view_start;  /* uint32[V+1]: first sorted visible entry of each view */
  size_t gauss_list;  /* uint32[N]: Gaussians g with a non-empty box in at least one view */
  size_t tile_count;  /* uint32[V*T]: pairs per tile, T = ceil(W/16) * ceil(H/16) */
  size_t tile_start;  /* uint32[V*T]: first pair of each tile in the sorted order */
  size_t bucket_count;  /* uint32[B]: row items (Gaussian, tile row of its box) per bucket */
  size_t bucket_start;  /* uint32[B] */
  size_t unit_first_e;  /* uint32[V+1]: first entry unit of each view */
  size_t unit_seg_e;    /* uint32[E/256 + V]: view of each entry unit */
  size_t unit_cnt_e;    /* uint32[ceil(H/16)][E/256 + V]: row items per tile row of each entry unit */
  size_t unit_first_r;  /* uint32[B+1]: first row unit of each bucket */
  size_t unit_seg_r;    /* uint32[cap/128 + B]: bucket of each row unit */
  size_t unit_cnt_r;    /* uint32[ceil(W/16)][cap/128 + B]: pairs per tile of each row unit */
  size_t row_items;   /* uint32[cap]: entry of each row item, grouped by bucket, in (depth key, index) order */
  size_t row_span;    /* uint32[cap]: kept tile columns of each row item */
  size_t sorted_ids;  /* uint32[cap]: Gaussian index of each pair, sorted by (tile, depth key, index) */
  size_t view_stats;  /* float[V][4]: per-view loss accumulators and valid-depth counts */
  size_t work_fill;   /* uint32[64]: items in each of the blend backward's 64 work classes */
  size_t work_lists;  /* uint32[64][V*T]: (view, tile) items of each work class; class c holds the tiles
                         whose longest contributor prefix w has floor(6 log2(w + 1)) = c (63: or more) */
  size_t total;       /* bytes */
} gs_layout;

/* Workspace bytes and layout for n Gaussians, a batch geometry and a pair
 * capacity.  Valid sizes: 1 <= n < 2^31, 1 <= pair_capacity < 2^31 (an empty
 * map has nothing to project: its image is the background, which the caller
 * fills without the library).  Return 0 / GS_ERR_ARG on invalid sizes, 0 /
 * GS_ERR_UNSUPPORTED when n_views * n >= 2^30 or n_views * T >= 2^31. */
size_t gs_workspace_size(int64_t n, const gs_frame* frame, int64_t pair_capacity);
gs_status gs_workspace_layout(int64_t n, const gs_frame* frame, int64_t pair_capacity, gs_layout* out);

/* Copy the workspace status word and pairs-needed counter to the host
 * (synchronous on the stream).  status_out: GS_OK, or GS_ERR_CAPACITY when the
 * last gs_bin_sort needed more than pair_capacity pairs (needed in
 * pairs_needed_out; render outputs of that batch are then invalid). */
gs_status gs_read_status(const gs_workspace* ws, gs_stream_t stream, int32_t* status_out, int64_t* pairs_needed_out);

/* Projection, colour and tile culling (the equations for mu_hat, mu' and
 * Sigma' before Eq. alpha; SH colour after Eq. rendered_opacity; Sec. "Fast
 * Tile-based Culling").  Per (view, Gaussian): mean2d, conic, opacity,
 * colour, depth, tile box, and the per-tile pair counts.  cams_dev: device
 * array of frame->n_views cameras.  Clears the workspace status and the 2D
 * adjoints of every projected Gaussian. */
gs_status gs_project(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg, const gs_workspace* ws,
                     gs_stream_t stream);

/* Binning and sorting: the visible (view, Gaussian) entries sorted once by
 * (view, depth key bits, Gaussian index), then stable scatters into (view,
 * tile row) buckets and into the tile bins of the kept (Gaussian, tile)
 * pairs, so each tile's Gaussians come out in (depth key, index) order, the
 * order of a sort on 64-bit (tile, depth) keys; tile ranges from the per-tile
 * counts.  On overflow the status word becomes GS_ERR_CAPACITY and the later
 * calls of the batch do nothing. */
gs_status gs_bin_sort(const gs_workspace* ws, gs_stream_t stream);

/* Front-to-back compositing per 16x16 tile (Eq. alpha, Eq. rendered_rgb,
 * rendered_depth, rendered_opacity): alpha = min(alpha_max, o exp(-q/2)),
 * skipped below alpha_min, stop before T would fall below t_min.  Outputs:
 * rgb [V][3][H][W] (with background), depth [V][H][W] (sum d alpha T, not
 * normalised), opac [V][H][W] (= 1 - T_final), t_final [V][H][W], n_contrib
 * [V][H][W] (1 + position in the tile list of the last blended Gaussian,
 * 0 if none).  Any output pointer except t_final and n_contrib may be NULL. */
gs_status gs_render_fwd(const gs_config* cfg, const gs_workspace* ws, float* rgb, float* depth, float* opac,
                        float* t_final, uint32_t* n_contrib, gs_stream_t stream);

/* Work counters of the compositing (measurement support; no counterpart in
 * the paper): runs the front-to-back compositing of gs_render_fwd over the
 * workspace's tile lists without writing an image and sets, per view,
 * counts_dev[3v] = number of (pixel, tile-list position) evaluations up to
 * each pixel's last blended Gaussian (the sum of gs_render_fwd's n_contrib),
 * counts_dev[3v + 1] = how many of them were blended (the others were
 * skipped below alpha_min) and counts_dev[3v + 2] = the tile-list positions
 * the pixels test (each up to and including the Gaussian at which it stops,
 * else its tile's whole list: the evaluations the forward cannot avoid).
 * counts_dev: device uint64 [V][3], 8-byte aligned, overwritten. */
gs_status gs_blend_counts(const gs_config* cfg, const gs_workspace* ws, uint64_t* counts_dev, gs_stream_t stream);

/* Backward pass (Eq. depth_loss back through Eq. rendered_* and the
 * projection).  Pixel adjoints are the fused loss (tgt_rgb != NULL):
 *   L_v = w_rgb mean_{3HW} |C^ - C| + w_depth / |M_d| sum_{D_s>0, O^>0} |D^/O^ - D_s|,
 *   |M_d| = #(D_s > 0) per view, L = sum_v L_v, sign(0) = 0,
 * plus the caller's dL/dC^ [V][3][H][W], dL/dD^ [V][H][W], dL/dO^ [V][H][W]
 * where given (any of the three may be NULL = zero; with tgt_rgb == NULL they
 * are the whole adjoint, e.g. of an autograd graph; with it they add further
 * loss terms such as gs_dssim's gradient).  Recomputes each
 * pixel's blending state back to front from t_final and n_contrib.  The
 * blend stage walks a work list of the batch's (view, tile) items, longest
 * first: each tile goes into one of 64 classes by its longest contributor
 * prefix (the maximum of its pixels' n_contrib), and CTA b of the one launch
 * over all views takes item b of the classes' items, longest class first.  The
 * order only schedules the work: any order gives the same gradients up to
 * the summation order of float atomics.
 * Gradients are ADDED to grad_* (caller zeroes them): grad_mean [3][N],
 * grad_log_scale [3][N], grad_quat [4][N], grad_logit_opacity [N],
 * grad_sh_dc [3][N], grad_sh_rest [K-1][3][N] (FP32 even for BF16 SH; may be
 * NULL when sh_degree == 0), grad_pose [V][6] = dL/d(rho, theta) of
 * T_v Exp(xi) (may be NULL), loss_out [V] (may be NULL; added to).  The six
 * parameter-gradient pointers may also all be NULL when grad_pose is given:
 * the pose gradient alone (camera tracking with the map fixed). */
gs_status gs_render_bwd(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg, const gs_workspace* ws,
                        const float* rgb, const float* depth, const float* opac, const float* t_final,
                        const uint32_t* n_contrib, const float* tgt_rgb, const float* tgt_depth, float w_rgb,
                        float w_depth, const float* dl_drgb, const float* dl_ddepth, const float* dl_dopac,
                        float* grad_mean, float* grad_log_scale, float* grad_quat, float* grad_logit_opacity,
                        float* grad_sh_dc, float* grad_sh_rest, float* grad_pose, float* loss_out,
                        gs_stream_t stream);

/* gs_render_bwd with the fused loss's colour targets given as the camera's
 * 8-bit images: tgt_rgb8 [V][3][H][W] uint8 (device; required), target value
 * c / 255 correctly rounded, which is exactly what gs_unpack_keyframes writes,
 * so the gradients and loss are those of gs_render_bwd on the unpacked planes.
 * The loss reads 3 bytes per pixel instead of 12, and no FP32 colour plane is
 * written first.  Every other argument, the work and the errors are
 * gs_render_bwd's. */
gs_status gs_render_bwd_rgb8(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                             const gs_workspace* ws, const float* rgb, const float* depth, const float* opac,
                             const float* t_final, const uint32_t* n_contrib, const uint8_t* tgt_rgb8,
                             const float* tgt_depth, float w_rgb, float w_depth, const float* dl_drgb,
                             const float* dl_ddepth, const float* dl_dopac, float* grad_mean, float* grad_log_scale,
                             float* grad_quat, float* grad_logit_opacity, float* grad_sh_dc, float* grad_sh_rest,
                             float* grad_pose, float* loss_out, gs_stream_t stream);

/* Per-Gaussian backward (Sec. "Per-Gaussian Backpropagation"), an
 * alternative to the pixel-parallel blend backward inside gs_render_bwd with
 * the same results: the depth-sorted Gaussians of each tile are cut into
 * buckets of 32, one warp lane per Gaussian, and the tile's pixels stream
 * through the lanes carrying their transmittance, so each Gaussian's adjoints
 * are summed in registers and added once per (Gaussian, tile).  The state at
 * each bucket's start is checkpointed by the forward.
 *   gs_bucket_workspace_size: bytes of the caller's device buffer for the
 *     checkpoints (5 floats per pixel per bucket, sized for the workspace's
 *     pair capacity); 0 on an invalid workspace.
 *   gs_render_fwd_checkpointed: gs_render_fwd, plus the checkpoints written
 *     into bucket_ws (device, 256-byte aligned).
 *   gs_render_bwd_buckets: gs_render_bwd with the same arguments and
 *     outputs, reading the checkpoints of the gs_render_fwd_checkpointed call
 *     of the same batch; rgb and depth (that call's outputs) are required. */
size_t gs_bucket_workspace_size(const gs_workspace* ws);
gs_status gs_render_fwd_checkpointed(const gs_config* cfg, const gs_workspace* ws, float* rgb, float* depth,
                                     float* opac, float* t_final, uint32_t* n_contrib, void* bucket_ws,
                                     gs_stream_t stream);
gs_status gs_render_bwd_buckets(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                                const gs_workspace* ws, const float* rgb, const float* depth, const float* opac,
                                const float* t_final, const uint32_t* n_contrib, const float* tgt_rgb,
                                const float* tgt_depth, float w_rgb, float w_depth, const float* dl_drgb,
                                const float* dl_ddepth, const float* dl_dopac, float* grad_mean,
                                float* grad_log_scale, float* grad_quat, float* grad_logit_opacity,
                                float* grad_sh_dc, float* grad_sh_rest, float* grad_pose, float* loss_out,
                                const void* bucket_ws, gs_stream_t stream);

/* Pose Jacobian rows (Eq. 3dgs_jacobi, right perturbation T Exp(xi),
 * xi = (rho, theta)): for n_pix listed pixels per view (pix_idx [V][n_pix],
 * linear index y*W + x, device), J [V][n_pix][3][6] = dC^/dxi by forward-mode
 * tangents through projection, SH colour and compositing, and the rendered
 * colour at those pixels in rgb_out [V][n_pix][3] (may be NULL).  Needs the
 * t_final/n_contrib of gs_render_fwd for the same batch. */
gs_status gs_pose_jacobian(const gs_map* map, const gs_camera* cams_dev, const gs_config* cfg,
                           const gs_workspace* ws, const int32_t* pix_idx, int32_t n_pix, float* J, float* rgb_out,
                           gs_stream_t stream);

/* D-SSIM term of the mapping loss (Sec. "Map Optimization") and of the
 * tracking loss (Eq. tracking_loss): per view, D = 1 - mean SSIM(img, tgt)
 * over its 3 channels and H x W pixels, SSIM of Wang et al. under an 11 x 11
 * Gaussian window (sigma 1.5, zero padding, C1 = 1e-4, C2 = 9e-4; the paper
 * takes the term from 3D Gaussian Splatting), computed with separable filters
 * (Sec. "Additional Strategies" (c)).  img, tgt: device [V][3][H][W] FP32.
 * Adds weight * D_v to loss[v] (loss may be NULL) and weight * dD_v/dimg to
 * dl_dimg [V][3][H][W] (may be NULL; e.g. the buffer later passed to
 * gs_render_bwd as dl_drgb).  scratch: caller-owned device buffer of
 * gs_dssim_scratch_bytes(V, H, W) bytes, 256-byte aligned, overwritten.
 * With W % 4 == 0 and 16-byte aligned img, tgt and dl_dimg the tiles are
 * staged by TMA, otherwise element by element (same results, bit for bit).
 * GS_ERR_ARG for missing pointers or sizes, GS_ERR_UNSUPPORTED for more than
 * 21845 views.  A tile copy whose bounded (1 s) wait runs out, which is not
 * expected, leaves NaN in the view's loss or the tile's dl_dimg. */
size_t gs_dssim_scratch_bytes(int32_t n_views, int32_t height, int32_t width);
gs_status gs_dssim(const float* img, const float* tgt, int32_t n_views, int32_t height, int32_t width, float weight,
                   float* loss, float* dl_dimg, void* scratch, gs_stream_t stream);

/* Camera tracking with the map fixed (Sec. "Camera Factor (Option 2)": N_t
 * Adam iterations on the pose for the loss of Eq. tracking_loss).  The pose
 * of view v is the right perturbation T_v = T0_v Exp(xi_v) of an initial
 * world-to-camera transform, xi = (rho, theta) translation first, the
 * convention of gs_render_bwd's grad_pose.
 * gs_pose_apply: cams_out[v] = cams0[v] with R, t replaced by those of
 * T0_v Exp(xi_v) (Rodrigues rotation, V-matrix translation); all device
 * pointers, xi [V][6].  gs_adam_pose: one Adam step (Kingma and Ba, bias
 * corrected) on xi [V][6] with gradient grad [V][6] (cleared afterwards, for
 * the next gs_render_bwd to add into), first/second moments m, v [V][6] and a
 * device step counter (int32, start at 0); lr per component of xi.  With
 * loss_dev [V] (the loss at the current xi, e.g. gs_render_bwd's loss_out),
 * best_loss_dev [V] (start at +inf) and best_xi_dev [V][6] all given, the
 * iterate of lowest loss so far is kept per view (all three NULL: not kept). */
typedef struct {
  float lr[6];
  float beta1, beta2, eps;
} gs_adam_config;
gs_status gs_pose_apply(const gs_camera* cams0_dev, const float* xi_dev, int32_t n_views, gs_camera* cams_out_dev,
                        gs_stream_t stream);
gs_status gs_adam_pose(float* xi_dev, float* grad_dev, float* m_dev, float* v_dev, int32_t* step_dev,
                       int32_t n_views, const gs_adam_config* cfg, const float* loss_dev, float* best_loss_dev,
                       float* best_xi_dev, gs_stream_t stream);

/* Photometric residual of camera factor option 2 (Sec. "Camera Factor
 * (Option 2)", Eq. map_optimize_pose): r = Log(T(t) T~^-1), with T(t) the
 * camera-to-world pose of the continuous-time trajectory at the frame's time
 * and T~ the pose the tracker optimised.  The library's cameras are
 * world-to-camera (A = T(t)^-1 in cams_traj_dev, B = T~^-1 in cams_opt_dev,
 * device arrays of n_views), so r_v = Log(A_v^-1 B_v): the twist (rho, theta),
 * translation first, with B_v = A_v Exp(r_v) under gs_pose_apply's Exp (for
 * B = gs_pose_apply(A, xi), r = xi).  Rotation angles are returned in [0, pi];
 * r_dev [V][6] FP32 device.  Only R and t of the cameras are read (not the
 * intrinsics).  GS_ERR_ARG for missing pointers or
 * n_views < 1. */
gs_status gs_pose_residual(const gs_camera* cams_traj_dev, const gs_camera* cams_opt_dev, int32_t n_views,
                           float* r_dev, gs_stream_t stream);

/* Sparse Adam over the map (Sec. "Additional Strategies" (a)): one Adam step
 * (Kingma and Ba, bias corrected with the device step counter step_dev,
 * advanced by one) on the Gaussians that took part in the workspace's last
 * gs_project batch (those with a tile box in some view); every other
 * Gaussian keeps its parameters and moments.  params / grads / m / v: FP32
 * SoA arrays in the gs_map layout (n = the workspace's Gaussian count; sh_rest
 * [K-1][3][N] may be NULL at sh_degree 0).  The gradients of the updated
 * Gaussians are cleared afterwards.  Learning rates per attribute; the paper
 * takes those of 3D Gaussian Splatting without decay. */
typedef struct {
  float* mean;
  float* log_scale;
  float* quat;
  float* logit_opacity;
  float* sh_dc;
  float* sh_rest;
} gs_param_set;
typedef struct {
  float lr_mean, lr_log_scale, lr_quat, lr_logit_opacity, lr_sh_dc, lr_sh_rest;
  float beta1, beta2, eps;
} gs_adam_map_config;
gs_status gs_sparse_adam(const gs_workspace* ws, int32_t sh_degree, const gs_param_set* params,
                         const gs_param_set* grads, const gs_param_set* m, const gs_param_set* v, int32_t* step_dev,
                         const gs_adam_map_config* cfg, gs_stream_t stream);

/* Keyframe unpacking (Sec. "Additional Strategies" (e): keyframes are moved
 * host -> device asynchronously; moving them compact keeps the copy behind
 * the kernels): rgb8 [V][3][H][W] 8-bit colour -> rgb [V][3][H][W] = c / 255;
 * if depth_idx is given, depth [V][H][W] is cleared and, for view v, the
 * entries depth_offsets[v] .. depth_offsets[v + 1] - 1 of (depth_idx = pixel
 * y W + x, depth_val) are written (indices outside the image are skipped).
 * All pointers device; depth_* may be NULL (colour only); rgb8 and rgb may
 * both be NULL when depth is given (depth only: the caller's loss reads the
 * 8-bit colour itself, as gs_render_bwd_rgb8 does).  GS_ERR_ARG when only one
 * of rgb8 / rgb is given or there is nothing to unpack. */
gs_status gs_unpack_keyframes(const uint8_t* rgb8_dev, int32_t n_views, int32_t height, int32_t width,
                              float* rgb_dev, const int32_t* depth_idx_dev, const float* depth_val_dev,
                              const int32_t* depth_offsets_dev, float* depth_dev, gs_stream_t stream);

/* Map expansion (Sec. "Expansion of Gaussian Map"): from the opacity map O
 * of a new keyframe (gs_render_fwd's opac, [H][W] of one view), the mask
 * O < tau (the paper: 0.99) marks newly observed regions, and only the points
 * projecting into it initialise new Gaussians.
 * gs_expand_select: points [3][P] world positions (device), cam_dev one
 * camera, cfg->near_z the near plane; writes the indices of the selected
 * points, ascending, to idx_out [P] and their number to *count_out (device
 * uint32).  A point is selected iff its depth exceeds near_z and the pixel
 * containing its projection (pixel i spans [i, i + 1)) lies in the image with
 * O < tau.  scratch: gs_expand_scratch_bytes(P) bytes, 256-byte aligned.
 * gs_expand_init: writes the *count_dev new Gaussians for idx_dev into dst at
 * [first, first + count) of FP32 SoA arrays holding n_dst Gaussians (entries
 * past n_dst are dropped): mean = the point, log-scales log(2 d / fx) (two
 * pixels across at depth d), quaternion (1, 0, 0, 0), opacity init_opacity,
 * SH DC from rgb_dev [3][P] in [0, 1] (colour = 0.5 + Y_00 DC), higher SH 0
 * (readings: the paper takes the initialisation from its predecessors). */
size_t gs_expand_scratch_bytes(int64_t n_points);
gs_status gs_expand_select(const float* points_dev, int64_t n_points, const gs_camera* cam_dev, const gs_config* cfg,
                           const float* opac_dev, int32_t height, int32_t width, float tau, void* scratch,
                           int32_t* idx_out, uint32_t* count_out, gs_stream_t stream);
gs_status gs_expand_init(const float* points_dev, const float* rgb_dev, int64_t n_points, const int32_t* idx_dev,
                         const uint32_t* count_dev, const gs_camera* cam_dev, int64_t first, const gs_param_set* dst,
                         int64_t n_dst, int32_t sh_degree, float init_opacity, gs_stream_t stream);

/* Spatial storage order of the map (measurement-driven; no counterpart in
 * the paper, which leaves the storage order open).  A view sees a fraction
 * of the Gaussians; ordered along a space-filling curve of their means, the
 * Gaussians a view or a tile sees are contiguous runs of the SoA arrays, so
 * the projection, the projection backward and the sparse Adam step
 * (Sec. "Additional Strategies" (a)) read and write whole sectors.
 *   gs_morton_scratch_bytes: bytes of the scratch buffer for n Gaussians
 *     (0 if n < 1 or n >= 2^30).
 *   gs_morton_order: perm_out [n] (device uint32) = the Gaussian indices
 *     sorted by the 30-bit Morton code of mean [3][n] (device FP32): per
 *     axis q = floor((m - lo) 1024 / (hi - lo)) clamped to [0, 1023] over the
 *     bounding box of the finite means (0 for a flat axis or a non-finite
 *     mean), x, y, z bits interleaved with x the most significant; equal
 *     codes in index order.  scratch: caller-owned device buffer of
 *     gs_morton_scratch_bytes(n) bytes, 256-byte aligned, overwritten.
 *   gs_permute_rows: dst[r][i] = src[r][perm[i]] for rows SoA rows of n
 *     elements of elem_bytes (2 or 4) bytes, e.g. each parameter array of a
 *     gs_param_set and the matching Adam moments; src and dst are distinct
 *     device buffers; an out-of-range perm[i] leaves dst[.][i] as it was.
 * The library keeps the caller's indexing everywhere: after permuting the
 * arrays, gradients, tile lists and outputs refer to the new order. */
size_t gs_morton_scratch_bytes(int64_t n);
gs_status gs_morton_order(const float* mean_dev, int64_t n, void* scratch, uint32_t* perm_out, gs_stream_t stream);
gs_status gs_permute_rows(const void* src_dev, void* dst_dev, int64_t rows, int64_t n, int32_t elem_bytes,
                          const uint32_t* perm_dev, gs_stream_t stream);

/* Forward render that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc - code running
 * inside a host framework that owns all device memory (an inference-engine
 * plugin, a middleware node that is handed fixed buffers) or a real-time loop
 * that cannot afford cudaMalloc's implicit device synchronisation.
 *
 * It does what gs_project + gs_bin_sort + gs_render_fwd do, with the same
 * kernels and outputs (rgb, depth, opac may be NULL; t_final and n_contrib
 * may not), but instead of a caller workspace it uses a file-scope device
 * array of GS_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU which loads the
 * library holds until the process exits.  The caller passes the map, the
 * device cameras, the batch geometry and every output; status_dev (device
 * int32) receives the batch's device status: GS_OK; GS_ERR_CAPACITY when the
 * pair buffer left in the array was too small (the images are then
 * background only: t_final 1, n_contrib 0); or GS_ERR_CUDA if the binning
 * found its per-tile counts inconsistent (an internal error, not expected).
 * Requests whose per-Gaussian and per-tile parts do not fit in the array are
 * rejected with GS_ERR_UNSUPPORTED before anything is enqueued.  With E =
 * V*N entries, T tiles per view and TY = ceil(H/16), TX = ceil(W/16), those
 * parts take about E*(131 + TY/64) bytes (projected records, tile boxes, 2D
 * adjoints, the visible list and its sort) + N*4 bytes (Gaussian list) +
 * V*T*264 bytes (per-tile counts and starts, the backward's work lists) + V*TY*(8 + 28*(1 + TX)) bytes
 * (per tile-row counts and the first binning units) + 6 KB; whatever is left
 * holds 12 + (1 + TX)/32 bytes per (Gaussian, tile) pair (about 16 B at
 * 1920 wide).  The call computes the split exactly with gs_workspace_size.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current) and caches it with the id
 * of the device's CUDA context; a call in another context (after
 * cudaDeviceReset, or once the primary context was released and created
 * again) looks it up anew.  Make the first call on a device, and the first
 * after such a reset, before any stream capture.  All calls share the one
 * array and it keeps the last call's contents (each call clears what must
 * start at zero): calls that overlap on the GPU - on two streams, or from two
 * host threads - race. */
#define GS_NOALLOC_SCRATCH_BYTES (64u << 20)
gs_status gs_render_fwd_noalloc(const gs_map* map, const gs_camera* cams_dev, const gs_frame* frame,
                                const gs_config* cfg, float* rgb, float* depth, float* opac, float* t_final,
                                uint32_t* n_contrib, int32_t* status_dev, gs_stream_t stream);

/* Per-kernel tracing (timing support; no counterpart in the paper).  While
 * active, each kernel the library launches is bracketed by
 * cudaEventRecord(events[2k]) / cudaEventRecord(events[2k+1]) on its stream,
 * k = 0, 1, ... in launch order, and kernel_ids[k] (may be NULL) receives the
 * kernel's id (see gs_kernel_name).  events: caller-created cudaEvent_t
 * handles, 2 * capacity of them, owned by the caller; launches beyond
 * capacity are counted but not recorded.  gs_trace_stop ends tracing and
 * returns the number of launches seen.  Drive the library from one host
 * thread while tracing. */
gs_status gs_trace_start(void* const* events, int32_t capacity, int32_t* kernel_ids);
int32_t gs_trace_stop(void);
const char* gs_kernel_name(int32_t id);

/* Static description of a status code. */
const char* gs_status_str(gs_status s);

/* Library version string ("gsb300 <major>.<minor>"). */
const char* gs_version(void);

/* Test support (no counterpart in the paper): the library's only device wait
 * is the radix sort's look-back of a tile on the tiles before it (binning),
 * bounded at 65536 polls, after which the sort's error word becomes
 * GS_ERR_TIMEOUT and the pass goes on writing only in-range slots.
 * gs_sort_wait_probe runs one pass of that sort on one CTA over a synthetic
 * array of 4096 keys held in scratch_dev (caller-owned device memory of at
 * least gs_sort_wait_probe_bytes() bytes, 16-byte aligned, overwritten).
 * skip_first_tile != 0 starts the pass's tile tickets at 1, so no CTA ever
 * takes tile 0 and the wait of tile 1 on it runs out (tens of milliseconds);
 * otherwise the pass is an ordinary stable sort by the keys' low byte.  The
 * pass's error word (GS_OK or GS_ERR_TIMEOUT) is copied to *status_dev
 * (device int32).  Returns GS_ERR_ARG for a NULL or short or misaligned
 * buffer; asynchronous on the stream otherwise. */
size_t gs_sort_wait_probe_bytes(void);
gs_status gs_sort_wait_probe(void* scratch_dev, size_t scratch_bytes, int32_t skip_first_tile, int32_t* status_dev,
                             gs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
