"""ctypes binding of ``libgsb300.so`` (argument marshalling only).

The entry points keep the C names of ``include/gs.h``.  Loading fails loudly
when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgsb300.so")

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED = range(7)
GS_NOALLOC_SCRATCH_BYTES = 64 << 20  # size of gs_render_fwd_noalloc's device array

EXPORTED = ("gs_workspace_size", "gs_workspace_layout", "gs_read_status", "gs_project", "gs_bin_sort",
            "gs_render_fwd", "gs_blend_counts", "gs_render_bwd", "gs_render_bwd_rgb8", "gs_bucket_workspace_size",
            "gs_render_fwd_checkpointed", "gs_render_bwd_buckets", "gs_pose_jacobian", "gs_render_fwd_noalloc",
            "gs_dssim_scratch_bytes", "gs_dssim", "gs_unpack_keyframes", "gs_pose_apply", "gs_pose_residual",
            "gs_adam_pose", "gs_sparse_adam", "gs_expand_scratch_bytes", "gs_expand_select", "gs_expand_init",
            "gs_morton_scratch_bytes", "gs_morton_order", "gs_permute_rows", "gs_sort_wait_probe_bytes",
            "gs_sort_wait_probe", "gs_trace_start", "gs_trace_stop", "gs_kernel_name", "gs_status_str", "gs_version")


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float)]


class gs_map(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("sh_bf16", C.c_int32),
                ("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("logit_opacity", C.c_void_p), ("sh_dc", C.c_void_p), ("sh_rest", C.c_void_p)]


class gs_frame(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("width", C.c_int32), ("height", C.c_int32)]


class gs_config(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float), ("near_z", C.c_float),
                ("dilation", C.c_float), ("fov_clamp", C.c_float), ("bg", C.c_float * 3)]


class gs_workspace(C.Structure):
    _fields_ = [("ptr", C.c_void_p), ("n", C.c_int64), ("pair_capacity", C.c_int64), ("frame", gs_frame)]


class gs_layout(C.Structure):
    _fields_ = [(k, C.c_size_t) for k in ("counters", "records", "rects", "adjoints", "visible", "vis_key", "sort_key",
                                          "sort_val", "radix_status", "view_start", "gauss_list", "tile_count",
                                          "tile_start", "bucket_count", "bucket_start", "unit_first_e", "unit_seg_e",
                                          "unit_cnt_e", "unit_first_r", "unit_seg_r", "unit_cnt_r", "row_items",
                                          "row_span", "sorted_ids", "view_stats", "work_fill",
                                          "work_lists", "total")]


class gs_adam_config(C.Structure):
    _fields_ = [("lr", C.c_float * 6), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class gs_param_set(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest")]


class gs_adam_map_config(C.Structure):
    _fields_ = [(k, C.c_float) for k in ("lr_mean", "lr_log_scale", "lr_quat", "lr_logit_opacity", "lr_sh_dc",
                                         "lr_sh_rest", "beta1", "beta2", "eps")]


class GsError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {status_str(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2507_04004_b300.build`")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, F = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        L.gs_workspace_size.argtypes = [I64, C.POINTER(gs_frame), I64]
        L.gs_workspace_size.restype = C.c_size_t
        L.gs_workspace_layout.argtypes = [I64, C.POINTER(gs_frame), I64, C.POINTER(gs_layout)]
        L.gs_read_status.argtypes = [C.POINTER(gs_workspace), P, C.POINTER(I32), C.POINTER(I64)]
        L.gs_project.argtypes = [C.POINTER(gs_map), P, C.POINTER(gs_config), C.POINTER(gs_workspace), P]
        L.gs_bin_sort.argtypes = [C.POINTER(gs_workspace), P]
        L.gs_render_fwd.argtypes = [C.POINTER(gs_config), C.POINTER(gs_workspace), P, P, P, P, P, P]
        L.gs_blend_counts.argtypes = [C.POINTER(gs_config), C.POINTER(gs_workspace), P, P]
        L.gs_render_bwd.argtypes = ([C.POINTER(gs_map), P, C.POINTER(gs_config), C.POINTER(gs_workspace)]
                                    + [P] * 7 + [F, F] + [P] * 3 + [P] * 8 + [P])
        L.gs_render_bwd_rgb8.argtypes = L.gs_render_bwd.argtypes
        L.gs_bucket_workspace_size.argtypes = [C.POINTER(gs_workspace)]
        L.gs_bucket_workspace_size.restype = C.c_size_t
        L.gs_render_fwd_checkpointed.argtypes = [C.POINTER(gs_config), C.POINTER(gs_workspace)] + [P] * 7
        L.gs_render_bwd_buckets.argtypes = ([C.POINTER(gs_map), P, C.POINTER(gs_config), C.POINTER(gs_workspace)]
                                            + [P] * 7 + [F, F] + [P] * 3 + [P] * 8 + [P, P])
        L.gs_pose_jacobian.argtypes = [C.POINTER(gs_map), P, C.POINTER(gs_config), C.POINTER(gs_workspace), P, I32,
                                       P, P, P]
        L.gs_render_fwd_noalloc.argtypes = [C.POINTER(gs_map), P, C.POINTER(gs_frame), C.POINTER(gs_config),
                                            P, P, P, P, P, P, P]
        L.gs_render_fwd_noalloc.restype = I32
        L.gs_dssim_scratch_bytes.argtypes = [I32, I32, I32]
        L.gs_dssim_scratch_bytes.restype = C.c_size_t
        L.gs_dssim.argtypes = [P, P, I32, I32, I32, F, P, P, P, P]
        L.gs_pose_apply.argtypes = [P, P, I32, P, P]
        L.gs_pose_residual.argtypes = [P, P, I32, P, P]
        L.gs_unpack_keyframes.argtypes = [P, I32, I32, I32, P, P, P, P, P, P]
        L.gs_expand_scratch_bytes.argtypes = [I64]
        L.gs_expand_scratch_bytes.restype = C.c_size_t
        L.gs_expand_select.argtypes = [P, I64, P, C.POINTER(gs_config), P, I32, I32, F, P, P, P, P]
        L.gs_expand_init.argtypes = [P, P, I64, P, P, P, I64, C.POINTER(gs_param_set), I64, I32, F, P]
        L.gs_sparse_adam.argtypes = [C.POINTER(gs_workspace), I32] + [C.POINTER(gs_param_set)] * 4 + [
            P, C.POINTER(gs_adam_map_config), P]
        L.gs_adam_pose.argtypes = [P, P, P, P, P, I32, C.POINTER(gs_adam_config), P, P, P, P]
        L.gs_morton_scratch_bytes.argtypes = [I64]
        L.gs_morton_scratch_bytes.restype = C.c_size_t
        L.gs_morton_order.argtypes = [P, I64, P, P, P]
        L.gs_permute_rows.argtypes = [P, P, I64, I64, I32, P, P]
        L.gs_sort_wait_probe_bytes.argtypes = []
        L.gs_sort_wait_probe_bytes.restype = C.c_size_t
        L.gs_sort_wait_probe.argtypes = [P, C.c_size_t, I32, P, P]
        L.gs_trace_start.argtypes = [C.POINTER(C.c_void_p), I32, P]
        L.gs_trace_start.restype = I32
        L.gs_trace_stop.argtypes = []
        L.gs_trace_stop.restype = I32
        L.gs_kernel_name.argtypes = [I32]
        L.gs_kernel_name.restype = C.c_char_p
        L.gs_status_str.argtypes = [I32]
        L.gs_status_str.restype = C.c_char_p
        L.gs_version.restype = C.c_char_p
        for name in ("gs_read_status", "gs_project", "gs_bin_sort", "gs_render_fwd", "gs_blend_counts", "gs_render_bwd",
                     "gs_render_bwd_rgb8",
                     "gs_render_fwd_checkpointed", "gs_render_bwd_buckets",
                     "gs_pose_jacobian", "gs_workspace_layout", "gs_dssim", "gs_pose_apply", "gs_pose_residual", "gs_adam_pose",
                     "gs_sparse_adam", "gs_expand_select", "gs_expand_init", "gs_unpack_keyframes",
                     "gs_morton_order", "gs_permute_rows", "gs_sort_wait_probe"):
            getattr(L, name).restype = I32
        _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().gs_status_str(int(code)).decode()


def check(fn: str, code: int) -> None:
    if code != GS_OK:
        raise GsError(fn, code)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def gs_workspace_size(n: int, frame: gs_frame, pair_capacity: int) -> int:
    return int(lib().gs_workspace_size(int(n), C.byref(frame), int(pair_capacity)))


def gs_workspace_layout(n: int, frame: gs_frame, pair_capacity: int) -> gs_layout:
    L = gs_layout()
    check("gs_workspace_layout", lib().gs_workspace_layout(int(n), C.byref(frame), int(pair_capacity), C.byref(L)))
    return L


def gs_read_status(ws: gs_workspace, stream: int):
    s, p = C.c_int32(0), C.c_int64(0)
    check("gs_read_status", lib().gs_read_status(C.byref(ws), C.c_void_p(stream), C.byref(s), C.byref(p)))
    return int(s.value), int(p.value)


def gs_project(m: gs_map, cams, cfg: gs_config, ws: gs_workspace, stream: int) -> None:
    check("gs_project", lib().gs_project(C.byref(m), _ptr(cams), C.byref(cfg), C.byref(ws), C.c_void_p(stream)))


def gs_bin_sort(ws: gs_workspace, stream: int) -> None:
    check("gs_bin_sort", lib().gs_bin_sort(C.byref(ws), C.c_void_p(stream)))


def gs_render_fwd(cfg: gs_config, ws: gs_workspace, rgb, depth, opac, t_final, n_contrib, stream: int) -> None:
    check("gs_render_fwd", lib().gs_render_fwd(C.byref(cfg), C.byref(ws), _ptr(rgb), _ptr(depth), _ptr(opac),
                                               _ptr(t_final), _ptr(n_contrib), C.c_void_p(stream)))


def gs_blend_counts(cfg: gs_config, ws: gs_workspace, counts, stream: int) -> None:
    check("gs_blend_counts", lib().gs_blend_counts(C.byref(cfg), C.byref(ws), _ptr(counts), C.c_void_p(stream)))


def gs_render_bwd(m: gs_map, cams, cfg: gs_config, ws: gs_workspace, rgb, depth, opac, t_final, n_contrib,
                  tgt_rgb, tgt_depth, w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale,
                  grad_quat, grad_logit, grad_sh_dc, grad_sh_rest, grad_pose, loss, stream: int) -> None:
    check("gs_render_bwd", lib().gs_render_bwd(
        C.byref(m), _ptr(cams), C.byref(cfg), C.byref(ws), _ptr(rgb), _ptr(depth), _ptr(opac), _ptr(t_final),
        _ptr(n_contrib), _ptr(tgt_rgb), _ptr(tgt_depth), C.c_float(w_rgb), C.c_float(w_depth), _ptr(dl_drgb),
        _ptr(dl_ddepth), _ptr(dl_dopac), _ptr(grad_mean), _ptr(grad_log_scale), _ptr(grad_quat), _ptr(grad_logit),
        _ptr(grad_sh_dc), _ptr(grad_sh_rest), _ptr(grad_pose), _ptr(loss), C.c_void_p(stream)))


def gs_render_bwd_rgb8(m: gs_map, cams, cfg: gs_config, ws: gs_workspace, rgb, depth, opac, t_final, n_contrib,
                       tgt_rgb8, tgt_depth, w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale,
                       grad_quat, grad_logit, grad_sh_dc, grad_sh_rest, grad_pose, loss, stream: int) -> None:
    check("gs_render_bwd_rgb8", lib().gs_render_bwd_rgb8(
        C.byref(m), _ptr(cams), C.byref(cfg), C.byref(ws), _ptr(rgb), _ptr(depth), _ptr(opac), _ptr(t_final),
        _ptr(n_contrib), _ptr(tgt_rgb8), _ptr(tgt_depth), C.c_float(w_rgb), C.c_float(w_depth), _ptr(dl_drgb),
        _ptr(dl_ddepth), _ptr(dl_dopac), _ptr(grad_mean), _ptr(grad_log_scale), _ptr(grad_quat), _ptr(grad_logit),
        _ptr(grad_sh_dc), _ptr(grad_sh_rest), _ptr(grad_pose), _ptr(loss), C.c_void_p(stream)))


def gs_bucket_workspace_size(ws: gs_workspace) -> int:
    return int(lib().gs_bucket_workspace_size(C.byref(ws)))


def gs_render_fwd_checkpointed(cfg: gs_config, ws: gs_workspace, rgb, depth, opac, t_final, n_contrib, bucket_ws: int,
                               stream: int) -> None:
    check("gs_render_fwd_checkpointed", lib().gs_render_fwd_checkpointed(
        C.byref(cfg), C.byref(ws), _ptr(rgb), _ptr(depth), _ptr(opac), _ptr(t_final), _ptr(n_contrib),
        C.c_void_p(bucket_ws), C.c_void_p(stream)))


def gs_render_bwd_buckets(m: gs_map, cams, cfg: gs_config, ws: gs_workspace, rgb, depth, opac, t_final, n_contrib,
                          tgt_rgb, tgt_depth, w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, grad_mean, grad_log_scale,
                          grad_quat, grad_logit, grad_sh_dc, grad_sh_rest, grad_pose, loss, bucket_ws: int,
                          stream: int) -> None:
    check("gs_render_bwd_buckets", lib().gs_render_bwd_buckets(
        C.byref(m), _ptr(cams), C.byref(cfg), C.byref(ws), _ptr(rgb), _ptr(depth), _ptr(opac), _ptr(t_final),
        _ptr(n_contrib), _ptr(tgt_rgb), _ptr(tgt_depth), C.c_float(w_rgb), C.c_float(w_depth), _ptr(dl_drgb),
        _ptr(dl_ddepth), _ptr(dl_dopac), _ptr(grad_mean), _ptr(grad_log_scale), _ptr(grad_quat), _ptr(grad_logit),
        _ptr(grad_sh_dc), _ptr(grad_sh_rest), _ptr(grad_pose), _ptr(loss), C.c_void_p(bucket_ws),
        C.c_void_p(stream)))


def gs_pose_jacobian(m: gs_map, cams, cfg: gs_config, ws: gs_workspace, pix, n_pix: int, J, rgb, stream: int) -> None:
    check("gs_pose_jacobian", lib().gs_pose_jacobian(C.byref(m), _ptr(cams), C.byref(cfg), C.byref(ws), _ptr(pix),
                                                     int(n_pix), _ptr(J), _ptr(rgb), C.c_void_p(stream)))


def gs_dssim_scratch_bytes(n_views: int, height: int, width: int) -> int:
    return int(lib().gs_dssim_scratch_bytes(int(n_views), int(height), int(width)))


def gs_dssim(img, tgt, n_views: int, height: int, width: int, weight: float, loss, dl_dimg, scratch,
             stream: int) -> None:
    check("gs_dssim", lib().gs_dssim(_ptr(img), _ptr(tgt), int(n_views), int(height), int(width), float(weight),
                                     _ptr(loss), _ptr(dl_dimg), _ptr(scratch), C.c_void_p(stream)))


def gs_pose_apply(cams0, xi, n_views: int, cams_out, stream: int) -> None:
    check("gs_pose_apply", lib().gs_pose_apply(_ptr(cams0), _ptr(xi), int(n_views), _ptr(cams_out),
                                               C.c_void_p(stream)))


def gs_pose_residual(cams_traj, cams_opt, n_views: int, r, stream: int) -> None:
    check("gs_pose_residual", lib().gs_pose_residual(_ptr(cams_traj), _ptr(cams_opt), int(n_views), _ptr(r),
                                                     C.c_void_p(stream)))


def gs_adam_pose(xi, grad, m, v, step, n_views: int, cfg: "gs_adam_config", stream: int, loss=None,
                 best_loss=None, best_xi=None) -> None:
    check("gs_adam_pose", lib().gs_adam_pose(_ptr(xi), _ptr(grad), _ptr(m), _ptr(v), _ptr(step), int(n_views),
                                             C.byref(cfg), _ptr(loss), _ptr(best_loss), _ptr(best_xi),
                                             C.c_void_p(stream)))


def param_set(t) -> gs_param_set:
    """gs_param_set of an object with the six SoA tensors (GaussianMap or Grads)."""
    rest = getattr(t, "sh_rest")
    return gs_param_set(*(C.c_void_p(x.data_ptr()) if x is not None and x.numel() else None
                          for x in (t.mean, t.log_scale, t.quat, t.logit_opacity, t.sh_dc, rest)))


def gs_sparse_adam(ws: gs_workspace, sh_degree: int, params: gs_param_set, grads: gs_param_set, m: gs_param_set,
                   v: gs_param_set, step, cfg: gs_adam_map_config, stream: int) -> None:
    check("gs_sparse_adam", lib().gs_sparse_adam(C.byref(ws), int(sh_degree), C.byref(params), C.byref(grads),
                                                 C.byref(m), C.byref(v), _ptr(step), C.byref(cfg),
                                                 C.c_void_p(stream)))


def gs_unpack_keyframes(rgb8, n_views: int, height: int, width: int, rgb, depth_idx, depth_val, depth_offsets, depth,
                        stream: int) -> None:
    check("gs_unpack_keyframes", lib().gs_unpack_keyframes(_ptr(rgb8), int(n_views), int(height), int(width),
                                                           _ptr(rgb), _ptr(depth_idx), _ptr(depth_val),
                                                           _ptr(depth_offsets), _ptr(depth), C.c_void_p(stream)))


def gs_expand_scratch_bytes(n_points: int) -> int:
    return int(lib().gs_expand_scratch_bytes(int(n_points)))


def gs_expand_select(points, n_points: int, cam, cfg: gs_config, opac, height: int, width: int, tau: float, scratch,
                     idx, count, stream: int) -> None:
    check("gs_expand_select", lib().gs_expand_select(_ptr(points), int(n_points), _ptr(cam), C.byref(cfg),
                                                     _ptr(opac), int(height), int(width), float(tau),
                                                     _ptr(scratch), _ptr(idx), _ptr(count), C.c_void_p(stream)))


def gs_expand_init(points, rgb, n_points: int, idx, count, cam, first: int, dst: gs_param_set, n_dst: int,
                   sh_degree: int, init_opacity: float, stream: int) -> None:
    check("gs_expand_init", lib().gs_expand_init(_ptr(points), _ptr(rgb), int(n_points), _ptr(idx), _ptr(count),
                                                 _ptr(cam), int(first), C.byref(dst), int(n_dst), int(sh_degree),
                                                 float(init_opacity), C.c_void_p(stream)))


def gs_morton_scratch_bytes(n: int) -> int:
    return int(lib().gs_morton_scratch_bytes(int(n)))


def gs_morton_order(mean, n: int, scratch, perm, stream: int) -> None:
    check("gs_morton_order", lib().gs_morton_order(_ptr(mean), int(n), _ptr(scratch), _ptr(perm),
                                                   C.c_void_p(stream)))


def gs_permute_rows(src, dst, rows: int, n: int, elem_bytes: int, perm, stream: int) -> None:
    check("gs_permute_rows", lib().gs_permute_rows(_ptr(src), _ptr(dst), int(rows), int(n), int(elem_bytes),
                                                   _ptr(perm), C.c_void_p(stream)))


def gs_render_fwd_noalloc(m: gs_map, cams, frame: gs_frame, cfg: gs_config, rgb, depth, opac, t_final, n_contrib,
                          status_dev, stream: int) -> int:
    """Allocation-free forward render; returns the synchronous status code."""
    return int(lib().gs_render_fwd_noalloc(C.byref(m), _ptr(cams), C.byref(frame), C.byref(cfg), _ptr(rgb),
                                           _ptr(depth), _ptr(opac), _ptr(t_final), _ptr(n_contrib),
                                           _ptr(status_dev), C.c_void_p(stream)))


def gs_trace_start(event_handles, kernel_ids) -> None:
    """event_handles: list of 2*capacity cudaEvent_t ints; kernel_ids: int32 numpy array of capacity."""
    arr = (C.c_void_p * len(event_handles))(*event_handles)
    _trace_keep[:] = [arr, kernel_ids]
    check("gs_trace_start", lib().gs_trace_start(arr, len(event_handles) // 2, kernel_ids.ctypes.data))


def gs_trace_stop() -> int:
    return int(lib().gs_trace_stop())


def gs_kernel_name(i: int) -> str:
    return lib().gs_kernel_name(int(i)).decode()


_trace_keep: list = []


def gs_version() -> str:
    return lib().gs_version().decode()


def gs_sort_wait_probe_bytes() -> int:
    return int(lib().gs_sort_wait_probe_bytes())


def gs_sort_wait_probe(scratch, skip_first_tile: bool, status, stream: int) -> None:
    check("gs_sort_wait_probe", lib().gs_sort_wait_probe(_ptr(scratch), int(scratch.numel() * scratch.element_size()),
                                                         1 if skip_first_tile else 0, _ptr(status),
                                                         C.c_void_p(stream)))
