"""Mapping step driven from host keyframes (public API used end to end).

arxiv 2507.04004, Sec. "Additional Strategies" (e): keyframe images and sparse
depth maps live in pinned host memory and are moved with asynchronous copies
on their own stream, so the upload of the next batch overlaps the kernels of
the current one.  Each :meth:`MappingStep.step` runs one fwd+bwd pass of the
rasterizer (projection, binning/sort, compositing, fused loss backward) over
a batch of keyframes and returns the per-view loss as a pinned host tensor.
"""
from __future__ import annotations

import torch

from .raster import GaussianMap, Grads, Rasterizer, RenderOut


class MappingStep:
    """Double-buffered host-to-device upload + one rasterizer pass per batch."""

    def __init__(self, rast: Rasterizer, gmap: GaussianMap, w_rgb: float, w_depth: float):
        self.rast, self.gmap, self.w_rgb, self.w_depth = rast, gmap, float(w_rgb), float(w_depth)
        V, H, W = rast.views, rast.height, rast.width
        dev = rast.device
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.slots = []
        for _ in range(2):
            self.slots.append(dict(
                rgb=torch.empty(V, 3, H, W, device=dev), depth=torch.empty(V, H, W, device=dev),
                cams=torch.empty(V, 16, device=dev), ready=torch.cuda.Event(), free=torch.cuda.Event()))
        f = dict(device=dev, dtype=torch.float32)
        self.out = RenderOut(torch.empty(V, 3, H, W, **f), torch.empty(V, H, W, **f), torch.empty(V, H, W, **f),
                             torch.empty(V, H, W, **f), torch.empty(V, H, W, dtype=torch.int32, device=dev))
        self.grads: Grads = rast.new_grads(gmap)
        self.loss_host = torch.empty(V, dtype=torch.float32, pin_memory=True)
        self.h2d_bytes = (V * 3 * H * W + V * H * W + V * 16) * 4
        self.d2h_bytes = V * 4
        self._next = 0

    def upload(self, host_rgb: torch.Tensor, host_depth: torch.Tensor, host_cams: torch.Tensor) -> dict:
        """Queue the copy of one batch (pinned host tensors) on the copy stream."""
        slot = self.slots[self._next]
        self._next ^= 1
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(slot["free"])
            slot["rgb"].copy_(host_rgb, non_blocking=True)
            slot["depth"].copy_(host_depth, non_blocking=True)
            slot["cams"].copy_(host_cams, non_blocking=True)
            slot["ready"].record(self.copy_stream)
        return slot

    def step(self, slot: dict) -> torch.Tensor:
        """One fwd+bwd pass on the current stream over an uploaded batch."""
        cur = torch.cuda.current_stream(self.rast.device)
        cur.wait_event(slot["ready"])
        g = self.grads
        for t in (g.mean, g.log_scale, g.quat, g.logit_opacity, g.sh_dc, g.sh_rest, g.pose, g.loss):
            t.zero_()
        self.rast.render(self.gmap, slot["cams"], check=False, out=self.out)
        self.rast.backward(self.gmap, slot["cams"], self.out, tgt_rgb=slot["rgb"], tgt_depth=slot["depth"],
                           w_rgb=self.w_rgb, w_depth=self.w_depth, grads=g)
        slot["free"].record(cur)
        self.loss_host.copy_(g.loss, non_blocking=True)
        return self.loss_host
