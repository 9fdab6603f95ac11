"""PyTorch face of the rasterizer: device memory, streams and autograd.

PyTorch only owns tensors and streams here; every step of the rasterizer
(projection, culling, binning, sort, compositing, backward, pose Jacobian)
runs in the CUDA kernels of ``libgsb300.so`` through :mod:`._native`.

Method: arxiv 2507.04004, Sec. "3D Gaussian Splatting Representation"
(projection, Eq. alpha, Eq. rendered_rgb / rendered_depth / rendered_opacity,
Eq. 3dgs_jacobi), Sec. "Fast Tile-based Culling" and Eq. depth_loss.
"""
from __future__ import annotations

from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np
import torch

from . import _native as N

DEFAULT_CONFIG = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, near_z=0.2, dilation=0.3, fov_clamp=1.3,
                      bg=(0.0, 0.0, 0.0))


def make_config(**over) -> N.gs_config:
    d = dict(DEFAULT_CONFIG)
    d.update(over)
    c = N.gs_config()
    for k in ("alpha_min", "alpha_max", "t_min", "near_z", "dilation", "fov_clamp"):
        setattr(c, k, float(d[k]))
    for i in range(3):
        c.bg[i] = float(d["bg"][i])
    return c


@dataclass
class GaussianMap:
    """Device-resident Gaussian parameters, structure of arrays (see gs.h)."""
    mean: torch.Tensor          # [3][N] f32
    log_scale: torch.Tensor     # [3][N] f32
    quat: torch.Tensor          # [4][N] f32 (w, x, y, z)
    logit_opacity: torch.Tensor  # [N] f32
    sh_dc: torch.Tensor         # [3][N] f32 or bf16
    sh_rest: torch.Tensor       # [K-1][3][N] f32 or bf16
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.logit_opacity.shape[0])

    @property
    def sh_bf16(self) -> bool:
        return self.sh_dc.dtype == torch.bfloat16

    @classmethod
    def from_host(cls, g, device="cuda", sh_bf16=False) -> "GaussianMap":
        """From a :class:`synth.GaussianMap` (numpy) or a dict of arrays."""
        d = g.as_dict() if hasattr(g, "as_dict") else g
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)
        sd = torch.bfloat16 if sh_bf16 else torch.float32
        return cls(f(d["mean"]), f(d["log_scale"]), f(d["quat"]), f(d["logit_opacity"]),
                   f(d["sh_dc"]).to(sd).contiguous(), f(d["sh_rest"]).to(sd).contiguous(), int(d["sh_degree"]))

    def permuted(self, perm: torch.Tensor) -> "GaussianMap":
        """The map with Gaussian i of the result = Gaussian perm[i] of this one."""
        p = lambda t: permute_rows(t, perm)
        return GaussianMap(p(self.mean), p(self.log_scale), p(self.quat), p(self.logit_opacity), p(self.sh_dc),
                           p(self.sh_rest), self.sh_degree)

    def spatially_ordered(self) -> tuple["GaussianMap", torch.Tensor]:
        """(the map in Morton order of its means, the permutation applied)."""
        perm = morton_order(self)
        return self.permuted(perm), perm

    def struct(self) -> N.gs_map:
        for t in (self.mean, self.log_scale, self.quat, self.logit_opacity, self.sh_dc, self.sh_rest):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("map tensors must be contiguous CUDA tensors")
        rest = self.sh_rest.data_ptr() if self.sh_degree > 0 else None
        return N.gs_map(self.n, self.sh_degree, 1 if self.sh_bf16 else 0, self.mean.data_ptr(),
                        self.log_scale.data_ptr(), self.quat.data_ptr(), self.logit_opacity.data_ptr(),
                        self.sh_dc.data_ptr(), rest)


def morton_order(gmap: "GaussianMap") -> torch.Tensor:
    """Permutation [N] (int32, device) sorting the Gaussians along the Morton
    curve of their means (gs_morton_order)."""
    dev = gmap.mean.device
    nbytes = N.gs_morton_scratch_bytes(gmap.n)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    perm = torch.empty(gmap.n, dtype=torch.int32, device=dev)
    N.gs_morton_order(gmap.mean, gmap.n, buf[off:off + nbytes], perm, torch.cuda.current_stream(dev).cuda_stream)
    return perm


def permute_rows(t: torch.Tensor, perm: torch.Tensor) -> torch.Tensor:
    """t[..., perm] for an SoA array whose last axis is the Gaussian index
    (gs_permute_rows), as a new tensor."""
    n = int(t.shape[-1])
    out = torch.empty_like(t)
    if t.numel():
        N.gs_permute_rows(t, out, t.numel() // n, n, t.element_size(), perm,
                          torch.cuda.current_stream(t.device).cuda_stream)
    return out


def cameras_tensor(cams, device="cuda") -> torch.Tensor:
    """[V][16] float32 rows in gs_camera layout (R row-major, t, fx, fy, cx, cy)."""
    rows = []
    for c in cams:
        rows.append(np.concatenate([np.asarray(c["R"], np.float32).reshape(9), np.asarray(c["t"], np.float32).reshape(3),
                                    np.array([c["fx"], c["fy"], c["cx"], c["cy"]], np.float32)]))
    return torch.as_tensor(np.stack(rows), device=device).contiguous()


@dataclass
class RenderOut:
    rgb: torch.Tensor        # [V][3][H][W]
    depth: torch.Tensor      # [V][H][W]
    opac: torch.Tensor       # [V][H][W]
    t_final: torch.Tensor    # [V][H][W]
    n_contrib: torch.Tensor  # [V][H][W] int32 (uint32 in the C ABI)


@dataclass
class Grads:
    mean: torch.Tensor
    log_scale: torch.Tensor
    quat: torch.Tensor
    logit_opacity: torch.Tensor
    sh_dc: torch.Tensor
    sh_rest: torch.Tensor
    pose: torch.Tensor       # [V][6]
    loss: torch.Tensor       # [V]
    flat: torch.Tensor | None = None  # one buffer holding all of the above (new_grads), else None

    def zero_(self) -> "Grads":
        """Clears every gradient: one fill of the shared buffer when there is one."""
        if self.flat is not None:
            self.flat.zero_()
        else:
            for t in (self.mean, self.log_scale, self.quat, self.logit_opacity, self.sh_dc, self.sh_rest,
                      self.pose, self.loss):
                t.zero_()
        return self


class Rasterizer:
    """Workspace owner for one batch geometry (n Gaussians, V views of W x H).

    The workspace keeps the projected Gaussians and tile lists of the last
    :meth:`render` / :meth:`project_and_sort` call, which :meth:`backward` and
    :meth:`pose_jacobian` reuse.  ``pair_capacity`` grows automatically when a
    checked call finds the pair buffer too small.

    ``backward``: "pixel" (default) runs the pixel-parallel blend backward;
    "bucket" the per-Gaussian one of Sec. "Per-Gaussian Backpropagation"
    (the forward then also writes its bucket checkpoints)."""

    def __init__(self, n: int, n_views: int, width: int, height: int, pair_capacity: int | None = None,
                 config: dict | None = None, device="cuda", backward: str = "pixel"):
        if backward not in ("pixel", "bucket"):
            raise ValueError("backward must be 'pixel' or 'bucket'")
        self.backward_mode = backward
        self._bucket_buf = None
        self.n, self.views, self.width, self.height = int(n), int(n_views), int(width), int(height)
        self.device = torch.device(device)
        self.cfg = make_config(**(config or {}))
        self.frame = N.gs_frame(self.views, self.width, self.height)
        self.capacity = int(pair_capacity or max(1 << 20, 4 * self.n * self.views))
        self._buf = None
        self.ws = None
        self.generation = 0
        self._alloc()

    def _alloc(self):
        size = N.gs_workspace_size(self.n, self.frame, self.capacity)
        if size == 0:
            raise ValueError("invalid workspace geometry")
        self._buf = torch.empty(size + 256, dtype=torch.uint8, device=self.device)
        base = self._buf.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.ws = N.gs_workspace(aligned, self.n, self.capacity, self.frame)
        self.layout = N.gs_workspace_layout(self.n, self.frame, self.capacity)
        self._base_off = aligned - base
        if self.backward_mode == "bucket":
            self._bucket_buf = None  # release before the new one is sized
            bsize = N.gs_bucket_workspace_size(self.ws)
            self._bucket_buf = torch.empty(bsize + 256, dtype=torch.uint8, device=self.device)
            self.bucket_ws = (self._bucket_buf.data_ptr() + 255) // 256 * 256

    @property
    def workspace_bytes(self) -> int:
        return int(self._buf.numel())

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _view(self, off: int, count: int, dtype) -> torch.Tensor:
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        start = self._base_off + off
        return self._buf[start:start + nbytes].view(dtype)

    # ---------------------------------------------------------------- state
    def status(self):
        """(status code, pairs needed) of the last binning (synchronises)."""
        return N.gs_read_status(self.ws, self._stream())

    def tile_lists(self):
        """(tile_start, tile_count, sorted_ids) int tensors of the last sort."""
        nt = self.views * ((self.width + 15) // 16) * ((self.height + 15) // 16)
        start = self._view(self.layout.tile_start, nt, torch.int32)
        count = self._view(self.layout.tile_count, nt, torch.int32)
        ids = self._view(self.layout.sorted_ids, self.capacity, torch.int32)
        return start, count, ids

    def records(self):
        """[V][N][12] float view of the projected records (mean2d, conic, ...)."""
        return self._view(self.layout.records, self.views * self.n * 12, torch.float32).view(self.views, self.n, 12)

    def rects(self):
        return self._view(self.layout.rects, self.views * self.n * 2, torch.int32).view(self.views, self.n, 2)

    # ---------------------------------------------------------------- calls
    def project_and_sort(self, gmap: GaussianMap, cams: torch.Tensor, check: bool = True) -> None:
        if gmap.n != self.n or cams.shape != (self.views, 16):
            raise ValueError("map / camera batch does not match the rasterizer geometry")
        m = gmap.struct()
        st = self._stream()
        for _ in range(4):
            N.gs_project(m, cams, self.cfg, self.ws, st)
            N.gs_bin_sort(self.ws, st)
            self.generation += 1
            if not check:
                return
            code, needed = self.status()
            if code == N.GS_OK:
                return
            if code != N.GS_ERR_CAPACITY:
                raise N.GsError("gs_bin_sort", code)
            self.capacity = int(needed * 1.25) + 1024
            self._alloc()
        raise RuntimeError("pair capacity did not converge")

    def render(self, gmap: GaussianMap, cams: torch.Tensor, check: bool = True, out: RenderOut | None = None
               ) -> RenderOut:
        self.project_and_sort(gmap, cams, check=check)
        V, H, W = self.views, self.height, self.width
        if out is None:
            f = dict(device=self.device, dtype=torch.float32)
            out = RenderOut(torch.empty(V, 3, H, W, **f), torch.empty(V, H, W, **f), torch.empty(V, H, W, **f),
                            torch.empty(V, H, W, **f), torch.empty(V, H, W, dtype=torch.int32, device=self.device))
        if self.backward_mode == "bucket":
            N.gs_render_fwd_checkpointed(self.cfg, self.ws, out.rgb, out.depth, out.opac, out.t_final, out.n_contrib,
                                         self.bucket_ws, self._stream())
        else:
            N.gs_render_fwd(self.cfg, self.ws, out.rgb, out.depth, out.opac, out.t_final, out.n_contrib,
                            self._stream())
        return out

    def new_grads(self, gmap: GaussianMap) -> Grads:
        """Zeroed gradient buffers, all views of one allocation (each part
        starting on a 256-byte boundary), so that Grads.zero_ clears them in
        one fill."""
        K = (gmap.sh_degree + 1) ** 2
        shapes = [(3, self.n), (3, self.n), (4, self.n), (self.n,), (3, self.n), (K - 1, 3, self.n),
                  (self.views, 6), (self.views,)]
        sizes = [int(np.prod(sh)) for sh in shapes]
        offs = [0]
        for sz in sizes:
            offs.append(offs[-1] + (sz + 63) // 64 * 64)
        flat = torch.zeros(offs[-1], device=self.device, dtype=torch.float32)
        parts = [flat[o:o + sz].view(*sh) for o, sz, sh in zip(offs, sizes, shapes)]
        return Grads(*parts, flat=flat)

    def backward(self, gmap: GaussianMap, cams: torch.Tensor, out: RenderOut, tgt_rgb=None, tgt_depth=None,
                 w_rgb: float = 1.0, w_depth: float = 0.0, dl_drgb=None, dl_ddepth=None, dl_dopac=None,
                 grads: Grads | None = None, pose: bool = True, params: bool = True) -> Grads:
        """Adds dL/dparams into ``grads`` (zeros when None) for the fused loss
        (``tgt_rgb`` given, FP32 or the 8-bit images; ``dl_*`` given as well add further loss terms) or
        the external pixel adjoints ``dl_*`` alone.  ``params=False``: the
        pose gradient (and loss) only, the map held fixed."""
        g = grads if grads is not None else self.new_grads(gmap)
        pg = (lambda t: t) if params else (lambda t: None)
        args = (gmap.struct(), cams, self.cfg, self.ws, out.rgb, out.depth, out.opac, out.t_final, out.n_contrib,
                tgt_rgb, tgt_depth, w_rgb, w_depth, dl_drgb, dl_ddepth, dl_dopac, pg(g.mean), pg(g.log_scale),
                pg(g.quat), pg(g.logit_opacity), pg(g.sh_dc), pg(g.sh_rest) if gmap.sh_degree > 0 else None,
                g.pose if pose else None, g.loss)
        if tgt_rgb is not None and tgt_rgb.dtype == torch.uint8:
            # 8-bit colour targets (c / 255) read by the fused loss itself
            if self.backward_mode == "bucket":
                raise ValueError("8-bit colour targets need the pixel-parallel backward")
            N.gs_render_bwd_rgb8(*args, self._stream())
        elif self.backward_mode == "bucket":
            N.gs_render_bwd_buckets(*args, self.bucket_ws, self._stream())
        else:
            N.gs_render_bwd(*args, self._stream())
        return g

    def pose_jacobian(self, gmap: GaussianMap, cams: torch.Tensor, pix: torch.Tensor):
        """J [V][n_pix][3][6] = dC/dxi and colour [V][n_pix][3] at ``pix``
        ([V][n_pix] int32 linear indices); uses the last projection."""
        V, n_pix = pix.shape
        J = torch.empty(V, n_pix, 3, 6, device=self.device, dtype=torch.float32)
        rgb = torch.empty(V, n_pix, 3, device=self.device, dtype=torch.float32)
        N.gs_pose_jacobian(gmap.struct(), cams, self.cfg, self.ws, pix.contiguous(), n_pix, J, rgb, self._stream())
        return J, rgb


class RasterizeFn(torch.autograd.Function):
    """(C^, D^, O^) = render(map, T_v Exp(xi_v)) with hand-written adjoints.

    ``xi`` is a [V][6] tensor that must hold zeros: its gradient is the
    right-perturbation pose gradient dL/dxi at xi = 0 (Eq. 3dgs_jacobi).
    """

    @staticmethod
    def forward(ctx, rast: Rasterizer, cams, xi, mean, log_scale, quat, logit_opacity, sh_dc, sh_rest, sh_degree):
        gmap = GaussianMap(mean.detach().contiguous(), log_scale.detach().contiguous(), quat.detach().contiguous(),
                           logit_opacity.detach().contiguous(), sh_dc.detach().contiguous(),
                           sh_rest.detach().contiguous(), int(sh_degree))
        out = rast.render(gmap, cams)
        ctx.rast, ctx.gmap, ctx.cams, ctx.out, ctx.gen = rast, gmap, cams, out, rast.generation
        ctx.mark_non_differentiable(out.t_final, out.n_contrib)
        return out.rgb, out.depth, out.opac

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_opac):
        rast, gmap = ctx.rast, ctx.gmap
        if rast.generation != ctx.gen:  # workspace reused since: project again (deterministic)
            rast.project_and_sort(gmap, ctx.cams)
        z = lambda t: None if t is None else t.contiguous()
        g = rast.backward(gmap, ctx.cams, ctx.out, dl_drgb=z(g_rgb), dl_ddepth=z(g_depth), dl_dopac=z(g_opac))
        sh_dc = g.sh_dc.to(gmap.sh_dc.dtype) if gmap.sh_bf16 else g.sh_dc
        sh_rest = g.sh_rest.to(gmap.sh_rest.dtype) if gmap.sh_bf16 else g.sh_rest
        return None, None, g.pose, g.mean, g.log_scale, g.quat, g.logit_opacity, sh_dc, sh_rest, None


def rasterize(rast: Rasterizer, cams, xi, gmap_params: dict, sh_degree: int):
    """Functional autograd entry: returns (rgb, depth, opacity)."""
    p = gmap_params
    return RasterizeFn.apply(rast, cams, xi, p["mean"], p["log_scale"], p["quat"], p["logit_opacity"], p["sh_dc"],
                             p["sh_rest"], sh_degree)


class DSSIM:
    """D-SSIM term (1 - mean SSIM per view, the 3DGS definition the paper's
    mapping and tracking losses use) on [V][3][H][W] images, through
    ``gs_dssim``; holds the scratch buffer for one image geometry."""

    def __init__(self, n_views: int, height: int, width: int, device="cuda"):
        self.shape = (int(n_views), int(height), int(width))
        nbytes = N.gs_dssim_scratch_bytes(*self.shape)
        self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self._buf.data_ptr()) % 256
        self.scratch = self._buf[off:off + nbytes]

    def __call__(self, img: torch.Tensor, tgt: torch.Tensor, weight: float = 1.0, loss: torch.Tensor | None = None,
                 dl_dimg: torch.Tensor | None = None) -> None:
        """Adds weight * D_v to loss[v] and weight * dD_v/dimg to dl_dimg (either may be None)."""
        V, H, W = self.shape
        if img.shape != (V, 3, H, W) or tgt.shape != img.shape:
            raise ValueError("image batch does not match the D-SSIM geometry")
        N.gs_dssim(img, tgt, V, H, W, weight, loss, dl_dimg, self.scratch,
                   torch.cuda.current_stream(img.device).cuda_stream)


class SparseAdam:
    """Sparse Adam on an FP32 map (Sec. "Additional Strategies" (a)) through
    ``gs_sparse_adam``: after a backward pass, one Adam step on the Gaussians
    the rasterizer's last projection saw, their gradients cleared.  Learning
    rates default to those of 3D Gaussian Splatting without decay (the paper's
    setting); ``spatial_scale`` multiplies the position rate (3DGS scales it by
    the scene extent)."""

    def __init__(self, gmap: GaussianMap, lr_mean: float = 1.6e-4, lr_log_scale: float = 5e-3,
                 lr_quat: float = 1e-3, lr_logit_opacity: float = 0.05, lr_sh_dc: float = 2.5e-3,
                 lr_sh_rest: float = 2.5e-3 / 20, betas=(0.9, 0.999), eps: float = 1e-15,
                 spatial_scale: float = 1.0):
        if gmap.sh_bf16:
            raise ValueError("sparse Adam updates FP32 maps")
        z = lambda t: torch.zeros_like(t)
        mk = lambda: SimpleNamespace(mean=z(gmap.mean), log_scale=z(gmap.log_scale), quat=z(gmap.quat),
                                     logit_opacity=z(gmap.logit_opacity), sh_dc=z(gmap.sh_dc),
                                     sh_rest=z(gmap.sh_rest))
        self.m, self.v = mk(), mk()
        self.step_count = torch.zeros(1, dtype=torch.int32, device=gmap.mean.device)
        self.cfg = N.gs_adam_map_config(lr_mean * spatial_scale, lr_log_scale, lr_quat, lr_logit_opacity, lr_sh_dc,
                                        lr_sh_rest, betas[0], betas[1], eps)

    def permute(self, perm: torch.Tensor) -> None:
        """Reorder the moments with the map (Gaussian i <- Gaussian perm[i])."""
        for st in (self.m, self.v):
            for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest"):
                setattr(st, k, permute_rows(getattr(st, k), perm))

    def step(self, gmap: GaussianMap, grads: Grads, rast: Rasterizer) -> None:
        N.gs_sparse_adam(rast.ws, gmap.sh_degree, N.param_set(gmap), N.param_set(grads), N.param_set(self.m),
                         N.param_set(self.v), self.step_count, self.cfg, rast._stream())


def expand_map(gmap: GaussianMap, points: torch.Tensor, colours: torch.Tensor, cam: torch.Tensor,
               opac: torch.Tensor, tau: float = 0.99, init_opacity: float = 0.1,
               config: dict | None = None) -> tuple[GaussianMap, torch.Tensor]:
    """Map expansion (Sec. "Expansion of Gaussian Map") for one keyframe:
    points / colours [3][P] (world, RGB in [0, 1]), cam [1][16], opac [H][W]
    (the keyframe's rendered opacity).  Returns the grown FP32 map (the old
    Gaussians first) and the indices of the points that became Gaussians."""
    if gmap.sh_bf16:
        raise ValueError("map expansion writes FP32 maps")
    dev = points.device
    P = int(points.shape[1])
    H, W = int(opac.shape[0]), int(opac.shape[1])
    st = torch.cuda.current_stream(dev).cuda_stream
    nbytes = N.gs_expand_scratch_bytes(P)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    idx = torch.empty(P, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    N.gs_expand_select(points, P, cam, make_config(**(config or {})), opac, H, W, tau, buf[off:off + nbytes], idx,
                       count, st)
    k = int(count.item())
    n0, n1 = gmap.n, gmap.n + k
    grow = lambda t: torch.cat([t, torch.empty(*t.shape[:-1], k, dtype=t.dtype, device=dev)], dim=-1).contiguous()
    out = GaussianMap(grow(gmap.mean), grow(gmap.log_scale), grow(gmap.quat), grow(gmap.logit_opacity),
                      grow(gmap.sh_dc), grow(gmap.sh_rest), gmap.sh_degree)
    if k:
        N.gs_expand_init(points, colours, P, idx, count, cam, n0, N.param_set(out), n1, gmap.sh_degree,
                         init_opacity, st)
    return out, idx[:k]
