"""Mapping step driven from host keyframes (public API used end to end).

arxiv 2507.04004, Sec. "Additional Strategies" (e): keyframe images and sparse
depth maps live in pinned host memory and are moved with asynchronous copies
on their own stream, so the upload of the next batch overlaps the kernels of
the current one.  A keyframe travels in the form a sensor delivers it: the
camera image as 8-bit RGB, the LiDAR depth map as its valid pixels only
((pixel index, depth) pairs, a few percent of the image).  The fused loss
reads the 8-bit images as they arrived (``gs_render_bwd_rgb8``);
``gs_unpack_keyframes`` expands the depth pairs into the FP32 depth map the
loss reads, as the first work of the batch's step on the compute stream.
Each :meth:`MappingStep.step` runs one fwd+bwd pass of the rasterizer
(projection, binning/sort, compositing, fused loss backward) over a batch of
keyframes and returns the per-view loss as a pinned host tensor; its device
work is replayed from one CUDA graph per upload slot (captured on first use),
so the ~30 launches and memsets of a step leave no gaps for the host to fill.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N
from .raster import GaussianMap, Grads, Rasterizer, RenderOut


class GraphStep:
    """A stream-ordered callable of fixed device buffers (no host reads, no
    allocation), replayed from a CUDA graph: run twice on a side stream, then
    captured.  replay() enqueues it on the current stream."""

    def __init__(self, fn, device=None, warmup: int = 2):
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()
        torch.cuda.current_stream(dev).wait_stream(side)

    def replay(self) -> None:
        self.graph.replay()


def pack_sparse_depth(depth: np.ndarray):
    """Dense depth maps [V][H][W] (0 = no depth) -> (idx [M] int32 pixel
    y W + x, val [M] float32, offsets [V + 1] int32), view by view in pixel
    order."""
    V = depth.shape[0]
    flat = np.asarray(depth, np.float32).reshape(V, -1)
    idx, val, offs = [], [], [0]
    for v in range(V):
        nz = np.flatnonzero(flat[v] > 0)
        idx.append(nz.astype(np.int32))
        val.append(flat[v, nz])
        offs.append(offs[-1] + nz.size)
    return np.concatenate(idx), np.concatenate(val), np.asarray(offs, np.int32)


@dataclass
class HostKeyframes:
    """One batch of V keyframes in pinned host memory.

    rgb8 [V][3][H][W] uint8; depth_idx [M] int32 (pixel y W + x within its
    view) and depth_val [M] float32, the valid LiDAR depths of view v being
    entries depth_offsets[v] .. depth_offsets[v + 1] - 1 (depth_offsets
    [V + 1] int32); cams [V][16] float32 (the rasterizer's camera records)."""
    rgb8: torch.Tensor
    depth_idx: torch.Tensor
    depth_val: torch.Tensor
    depth_offsets: torch.Tensor
    cams: torch.Tensor

    @staticmethod
    def from_dense(rgb8: np.ndarray, depth: np.ndarray, cams: torch.Tensor, pin: bool = True) -> "HostKeyframes":
        """Packs an 8-bit image batch and dense depth maps (0 = no depth)."""
        idx, val, offs = pack_sparse_depth(depth)
        host = lambda t: t.pin_memory() if pin else t
        arr = lambda a: host(torch.as_tensor(np.ascontiguousarray(a)))
        return HostKeyframes(arr(np.asarray(rgb8, np.uint8)), arr(idx), arr(val), arr(offs),
                             host(cams.to("cpu", torch.float32).contiguous()))

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size()
                   for t in (self.rgb8, self.depth_idx, self.depth_val, self.depth_offsets, self.cams))


class MappingStep:
    """Double-buffered host-to-device upload + one rasterizer pass per batch."""

    def __init__(self, rast: Rasterizer, gmap: GaussianMap, w_rgb: float, w_depth: float, graphs: bool = True):
        self.rast, self.gmap, self.w_rgb, self.w_depth = rast, gmap, float(w_rgb), float(w_depth)
        self.graphs = bool(graphs)
        # the pixel-parallel backward reads the 8-bit colour itself; the bucket
        # backward takes the FP32 planes, which the step then unpacks as well
        self.rgb8_loss = rast.backward_mode == "pixel"
        V, H, W = rast.views, rast.height, rast.width
        dev = rast.device
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.slots = []
        for _ in range(2):
            # the pair buffers hold a full image per view, so any depth map fits
            self.slots.append(dict(
                rgb8=torch.empty(V, 3, H, W, dtype=torch.uint8, device=dev),
                idx=torch.empty(V * H * W, dtype=torch.int32, device=dev),
                val=torch.empty(V * H * W, dtype=torch.float32, device=dev),
                offsets=torch.empty(V + 1, dtype=torch.int32, device=dev),
                rgb=None if self.rgb8_loss else torch.empty(V, 3, H, W, device=dev),
                depth=torch.empty(V, H, W, device=dev),
                cams=torch.empty(V, 16, device=dev), ready=torch.cuda.Event(), free=torch.cuda.Event()))
        f = dict(device=dev, dtype=torch.float32)
        self.out = RenderOut(torch.empty(V, 3, H, W, **f), torch.empty(V, H, W, **f), torch.empty(V, H, W, **f),
                             torch.empty(V, H, W, **f), torch.empty(V, H, W, dtype=torch.int32, device=dev))
        self.grads: Grads = rast.new_grads(gmap)
        self.loss_host = torch.empty(V, dtype=torch.float32, pin_memory=True)
        self.h2d_bytes = 0  # bytes of the last upload
        self.d2h_bytes = V * 4
        self._next = 0

    def upload(self, kf: HostKeyframes) -> dict:
        """Queue the copy of one batch (pinned host tensors, kept alive by the
        caller until the batch's step has run) on the copy stream.  The batch
        is unpacked by its step, on the compute stream: run on the copy stream,
        the unpacking's CTAs would share the SMs with the step's kernels and
        delay them by more than the unpacking takes on its own."""
        V, H, W = self.rast.views, self.rast.height, self.rast.width
        m = kf.depth_idx.numel()
        if tuple(kf.rgb8.shape) != (V, 3, H, W) or kf.depth_offsets.numel() != V + 1 or m > V * H * W:
            raise ValueError("keyframe batch does not match the rasterizer's views and image size")
        slot = self.slots[self._next]
        self._next ^= 1
        cs = self.copy_stream
        with torch.cuda.stream(cs):
            cs.wait_event(slot["free"])
            slot["rgb8"].copy_(kf.rgb8, non_blocking=True)
            slot["idx"][:m].copy_(kf.depth_idx, non_blocking=True)
            slot["val"][:m].copy_(kf.depth_val, non_blocking=True)
            slot["offsets"].copy_(kf.depth_offsets, non_blocking=True)
            slot["cams"].copy_(kf.cams, non_blocking=True)
            slot["ready"].record(cs)
        self.h2d_bytes = kf.nbytes()
        return slot

    def _work(self, slot: dict) -> None:
        V, H, W = self.rast.views, self.rast.height, self.rast.width
        # the depth map (and the colour planes only for the bucket backward: the
        # pixel-parallel one reads the 8-bit colour itself, gs_render_bwd_rgb8)
        rgb8 = None if self.rgb8_loss else slot["rgb8"]
        N.gs_unpack_keyframes(rgb8, V, H, W, slot["rgb"], slot["idx"], slot["val"], slot["offsets"], slot["depth"],
                              torch.cuda.current_stream(self.rast.device).cuda_stream)
        g = self.grads
        g.zero_()
        self.rast.render(self.gmap, slot["cams"], check=False, out=self.out)
        tgt = slot["rgb8"] if self.rgb8_loss else slot["rgb"]
        self.rast.backward(self.gmap, slot["cams"], self.out, tgt_rgb=tgt, tgt_depth=slot["depth"],
                           w_rgb=self.w_rgb, w_depth=self.w_depth, grads=g)

    def step(self, slot: dict) -> torch.Tensor:
        """One fwd+bwd pass on the current stream over an uploaded batch."""
        cur = torch.cuda.current_stream(self.rast.device)
        cur.wait_event(slot["ready"])
        if self.graphs:
            if "graph" not in slot:
                slot["graph"] = GraphStep(lambda: self._work(slot), self.rast.device)
            slot["graph"].replay()
        else:
            self._work(slot)
        slot["free"].record(cur)
        self.loss_host.copy_(self.grads.loss, non_blocking=True)
        return self.loss_host
