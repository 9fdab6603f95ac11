"""Camera tracking against a fixed Gaussian map (arxiv 2507.04004, Sec.
"Camera Factor (Option 2)"): for each frame, N_t Adam iterations on the pose
minimise Eq. tracking_loss, 1/2 L1 + 1/2 D-SSIM between the rendered and the
captured image, while the map stays fixed; the optimised pose feeds the
photometric constraint of Eq. map_optimize_pose.

A batch of frames is tracked together as the views of one rasterizer batch.
The pose of frame v is T0_v Exp(xi_v) (right perturbation, xi = (rho,
theta)); one iteration is

    cams = T0 Exp(xi)                         gs_pose_apply
    project, bin, sort, composite             gs_project, gs_bin_sort, gs_render_fwd
    dL/dC of 1/2 D-SSIM                       gs_dssim
    + fused 1/2 L1, back to the pose only     gs_render_bwd (no parameter gradients)
    Adam step on xi                           gs_adam_pose

and the N_t iterations are captured once as a CUDA graph and replayed per
batch.  After tracking, :meth:`PoseTracker.residual` forms the photometric
residual r = Log(T(t) T~^-1) of Eq. map_optimize_pose that the factor graph
consumes (gs_pose_residual).  All of it runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from .raster import DSSIM, GaussianMap, Grads, Rasterizer, RenderOut


class PoseTracker:
    """Tracks ``n_frames`` frames of ``width`` x ``height`` against ``gmap``.

    ``lr_trans`` / ``lr_rot``: Adam learning rates of rho and theta (the paper
    gives none; defaults are readings, stated with the tracker's tests)."""

    def __init__(self, gmap: GaussianMap, n_frames: int, width: int, height: int, iters: int = 30,
                 lr_trans: float = 3e-3, lr_rot: float = 3e-3, w_l1: float = 0.5, w_dssim: float = 0.5,
                 use_graph: bool = True, pair_capacity: int | None = None, device="cuda"):
        self.gmap, self.V, self.W, self.H = gmap, int(n_frames), int(width), int(height)
        self.iters, self.w_l1, self.w_dssim, self.use_graph = int(iters), float(w_l1), float(w_dssim), use_graph
        dev = torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        V, H, W = self.V, self.H, self.W
        f = dict(device=dev, dtype=torch.float32)
        self.rast = Rasterizer(gmap.n, V, W, H, pair_capacity=pair_capacity, device=dev)
        self.cams0 = torch.zeros(V, 16, **f)
        self.cams = torch.zeros(V, 16, **f)
        self.xi = torch.zeros(V, 6, **f)
        self.m = torch.zeros(V, 6, **f)
        self.s = torch.zeros(V, 6, **f)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.best_loss = torch.full((V,), float("inf"), **f)
        self.best_xi = torch.zeros(V, 6, **f)
        self.tgt = torch.zeros(V, 3, H, W, **f)
        self.dl = torch.zeros(V, 3, H, W, **f)
        self.out = RenderOut(torch.empty(V, 3, H, W, **f), torch.empty(V, H, W, **f), torch.empty(V, H, W, **f),
                             torch.empty(V, H, W, **f), torch.empty(V, H, W, dtype=torch.int32, device=dev))
        e = torch.empty(0, **f)
        self.grads = Grads(e, e, e, e, e, e, torch.zeros(V, 6, **f), torch.zeros(V, **f))
        self.loss_hist = torch.zeros(self.iters, V, **f)
        self.dssim = DSSIM(V, H, W, device=dev)
        lr = (ctypes.c_float * 6)(*([lr_trans] * 3 + [lr_rot] * 3))
        self.adam = N.gs_adam_config(lr, 0.9, 0.999, 1e-8)
        self.graph = None

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _iteration(self, it: int) -> None:
        st = self._stream()
        N.gs_pose_apply(self.cams0, self.xi, self.V, self.cams, st)
        self.rast.render(self.gmap, self.cams, check=False, out=self.out)
        self.dl.zero_()
        self.grads.loss.zero_()
        if self.w_dssim != 0.0:
            self.dssim(self.out.rgb, self.tgt, self.w_dssim, loss=self.grads.loss, dl_dimg=self.dl)
        self.rast.backward(self.gmap, self.cams, self.out, tgt_rgb=self.tgt, w_rgb=self.w_l1, w_depth=0.0,
                           dl_drgb=self.dl, grads=self.grads, params=False)
        self.loss_hist[it].copy_(self.grads.loss)
        N.gs_adam_pose(self.xi, self.grads.pose, self.m, self.s, self.step, self.V, self.adam, st,
                       loss=self.grads.loss, best_loss=self.best_loss, best_xi=self.best_xi)

    def _run(self) -> None:
        for it in range(self.iters):
            self._iteration(it)

    def _reset(self) -> None:
        self.xi.zero_()
        self.m.zero_()
        self.s.zero_()
        self.step.zero_()
        self.grads.pose.zero_()
        self.best_loss.fill_(float("inf"))
        self.best_xi.zero_()

    def _capture(self) -> None:
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin(capture_error_mode="thread_local")
            try:
                self._run()
            finally:
                g.capture_end()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = g

    def track(self, cams0: torch.Tensor, targets: torch.Tensor):
        """Optimise the poses of the batch: cams0 [V][16] (initial poses and
        intrinsics), targets [V][3][H][W].  Returns (xi [V][6], loss of each
        iteration [N_t][V]) as device tensors: xi is, per frame, the iterate of
        lowest loss among the N_t evaluated (the first is xi = 0), and the
        optimised pose of frame v is cams0_v Exp(xi_v)."""
        self.cams0.copy_(cams0)
        self.tgt.copy_(targets)
        self._reset()
        if self.graph is None:
            # size the pair buffer at the initial poses (with the rasterizer's headroom), first run eagerly
            self.rast.project_and_sort(self.gmap, self.cams0, check=True)
            self._run()
            if self.use_graph:
                self._reset()
                self._capture()
        if self.graph is not None:
            self.graph.replay()
        code, needed = self.rast.status()
        if code != N.GS_OK:
            # the poses moved into more pairs than the buffer holds: grow it, rerun eagerly, recapture next call
            self.rast.capacity = int(needed * 1.5) + 1024
            self.rast._alloc()
            self.graph = None
            self._reset()
            self._run()
            code, needed = self.rast.status()
            if code != N.GS_OK:
                raise N.GsError("track", code)
        return self.best_xi, self.loss_hist

    def optimised_cameras(self) -> torch.Tensor:
        """[V][16] cameras at the tracked poses cams0_v Exp(xi_v) of the last
        :meth:`track` call (the best iterate per frame)."""
        out = torch.empty_like(self.cams0)
        N.gs_pose_apply(self.cams0, self.best_xi, self.V, out, self._stream())
        return out

    def residual(self, cams_traj: torch.Tensor | None = None) -> torch.Tensor:
        """r [V][6] = Log(T(t) T~^-1) (Eq. map_optimize_pose, camera-to-world
        T(t), T~) as (rho, theta): ``cams_traj`` [V][16] holds the trajectory's
        poses T(t) as world-to-camera cameras (default: the initial poses of the
        last :meth:`track` call), T~ is the tracked pose."""
        a = self.cams0 if cams_traj is None else cams_traj.contiguous()
        r = torch.empty(self.V, 6, device=self.device, dtype=torch.float32)
        N.gs_pose_residual(a, self.optimised_cameras(), self.V, r, self._stream())
        return r
