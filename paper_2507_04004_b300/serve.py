"""Continuous-batching server for novel-view renders and tracking Jacobians.

Requests (a camera pose at some resolution; tracking requests add pixel
indices and target colours) arrive against one device-resident Gaussian map
(arxiv 2507.04004: novel-view rendering at a queried pose, Sec. "Video Frame
Interpolation"/"Rapid Mesh Reconstruction" use-cases; tracking with camera
factor option 2, Sec. "Camera Factor (Option 2)").  The server

* groups waiting requests by (kind, resolution) and packs up to ``max_views``
  of them into one multi-view launch of the rasterizer (views folded into the
  tile index, so every kernel runs once for the whole batch);
* admits a batch only while the workspaces of the batches in flight stay
  within ``mem_budget`` bytes (the sort buffers dominate a workspace);
* replays a CUDA graph captured per (kind, resolution, slot count) with the
  request cameras copied into the graph's camera buffer;
* runs batches on a pool of streams so that batches formed while others are
  on the GPU overlap with them, and resolves each request's future when its
  batch's completion event fires;
* creates a runner that is missing while batches are in flight on a builder
  thread (workspace allocation and graph capture take milliseconds), so the
  scheduler keeps launching meanwhile.

All rasterizer work runs in the CUDA kernels of ``libgsb300.so``.  A batch whose
pair buffer overflowed (device status word) is re-run eagerly with a larger
buffer and its graph re-captured.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as N
from .raster import GaussianMap, Rasterizer, RenderOut, cameras_tensor


# Bytes of a workspace that scale with its pair capacity (the sort buffers):
# 64-bit keys, 64-bit merge buffer, 32-bit sorted indices, 64-bit row items,
# 32-bit row spans.
SORT_BYTES_PER_PAIR = 8 + 8 + 4 + 8 + 4


@dataclass
class Request:
    kind: str                      # "render" or "jacobian"
    camera: dict                   # synth.camera(...) dict (pose + intrinsics + size)
    pix: np.ndarray | None = None  # jacobian: int32 linear pixel indices
    target: np.ndarray | None = None  # jacobian: [n_pix][3] target colours
    arrival: float = 0.0           # time.perf_counter() at submission (set by submit)
    launched: float = 0.0          # when its batch was launched
    done: float = 0.0
    future: Future = field(default_factory=Future)
    # streaming consumers: called with (request, result) on the scheduler
    # thread instead of storing the result in the future (resolved with None)
    on_result: object = None

    @property
    def key(self):
        c = self.camera
        npix = 0 if self.pix is None else len(self.pix)
        return (self.kind, int(c["width"]), int(c["height"]), npix)


def _slot_counts(max_views):
    s, out = 1, []
    while s <= max_views:
        out.append(s)
        s *= 2
    return out


class _Runner:
    """Workspace, buffers and (optionally) a captured graph for one
    (kind, resolution, slot count)."""

    def __init__(self, server, key, slots, capacity):
        kind, W, H, npix = key
        self.server, self.key, self.slots = server, key, slots
        dev = server.device
        self.rast = Rasterizer(server.gmap.n, slots, W, H, pair_capacity=capacity, device=dev)
        self.cams = torch.zeros(slots, 16, device=dev)
        f = dict(device=dev, dtype=torch.float32)
        self.out = RenderOut(torch.empty(slots, 3, H, W, **f), torch.empty(slots, H, W, **f),
                             torch.empty(slots, H, W, **f), torch.empty(slots, H, W, **f),
                             torch.empty(slots, H, W, dtype=torch.int32, device=dev))
        self.jac = kind == "jacobian"
        if self.jac:
            self.pix = torch.zeros(slots, npix, dtype=torch.int32, device=dev)
            self.J = torch.empty(slots, npix, 3, 6, **f)
            self.jrgb = torch.empty(slots, npix, 3, **f)
        self.host_cams = torch.empty(slots, 16, pin_memory=True)
        self.host_pix = torch.empty(slots, npix, dtype=torch.int32, pin_memory=True) if self.jac else None
        self.status = torch.zeros(2, dtype=torch.int32, device=dev)  # (status, pairs needed)
        self.host_status = torch.zeros(2, dtype=torch.int32, pin_memory=True)
        self.graph = None
        self.event = torch.cuda.Event()
        self.busy = False
        self.outputs = None
        self.bytes = SORT_BYTES_PER_PAIR * self.rast.capacity

    # -- the device work of one batch (captured once per runner)
    def _work(self):
        gm = self.server.gmap
        self.rast.project_and_sort(gm, self.cams, check=False)
        N.gs_render_fwd(self.rast.cfg, self.rast.ws, self.out.rgb, self.out.depth, self.out.opac,
                        self.out.t_final, self.out.n_contrib, torch.cuda.current_stream(self.server.device).cuda_stream)
        if self.jac:
            N.gs_pose_jacobian(gm.struct(), self.cams, self.rast.cfg, self.rast.ws, self.pix, self.pix.shape[1],
                               self.J, self.jrgb, torch.cuda.current_stream(self.server.device).cuda_stream)
        cnt = self.rast._view(self.rast.layout.counters, 2, torch.int32)
        self.status.copy_(cnt)

    def grow(self, pairs: int):
        """Re-allocate the workspace for ``pairs`` pairs and drop the graph."""
        self.rast.capacity = int(pairs)
        self.rast._alloc()
        self.bytes = SORT_BYTES_PER_PAIR * self.rast.capacity
        self.graph = None

    def capture(self, warm: bool = True):
        s = torch.cuda.Stream(device=self.server.device)
        if warm:
            with torch.cuda.stream(s):
                self._work()  # first run outside the capture (sets kernel attributes)
            s.synchronize()
        # capture_begin/end directly: the torch.cuda.graph context manager
        # synchronises the device and empties the allocator cache on entry,
        # which would stall every batch in flight
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin(capture_error_mode="thread_local")
            try:
                self._work()
            finally:
                g.capture_end()
            # the first launch of an instantiated graph uploads it to the device
            # (tens of milliseconds for these graphs): do it here, not on a request
            g.replay()
        s.synchronize()
        self.graph = g

    def launch(self, reqs, stream):
        """Copy inputs, run, copy each request's results into its own pinned
        host tensors (async; the tensors come from torch's pinned-memory cache
        and are handed to the caller without a further copy)."""
        n = len(reqs)
        for i, r in enumerate(reqs):
            self.host_cams[i] = torch.as_tensor(cameras_tensor([r.camera], device="cpu")[0])
            if self.jac:
                self.host_pix[i] = torch.as_tensor(r.pix)
        for i in range(n, self.slots):  # unused slots repeat the first camera
            self.host_cams[i] = self.host_cams[0]
            if self.jac:
                self.host_pix[i] = self.host_pix[0]
        with torch.cuda.stream(stream):
            self.cams.copy_(self.host_cams, non_blocking=True)
            if self.jac:
                self.pix.copy_(self.host_pix, non_blocking=True)
            if self.graph is not None and self.server.use_graphs:
                self.graph.replay()
            else:
                self._work()
            self.outputs = []
            for i in range(n):
                if self.jac:
                    J = torch.empty(self.J.shape[1:], pin_memory=True)
                    rgb = torch.empty(self.jrgb.shape[1:], pin_memory=True)
                    J.copy_(self.J[i], non_blocking=True)
                    rgb.copy_(self.jrgb[i], non_blocking=True)
                    self.outputs.append((J, rgb))
                else:
                    rgb = torch.empty(self.out.rgb.shape[1:], pin_memory=True)
                    dep = torch.empty(self.out.depth.shape[1:], pin_memory=True)
                    rgb.copy_(self.out.rgb[i], non_blocking=True)
                    dep.copy_(self.out.depth[i], non_blocking=True)
                    self.outputs.append((rgb, dep))
            self.host_status.copy_(self.status, non_blocking=True)
            self.event.record(stream)

    def results(self, reqs):
        out = []
        for r, (a, b) in zip(reqs, self.outputs):
            if self.jac:
                J, rgb = a.numpy(), b.numpy()
                res = rgb - (r.target if r.target is not None else 0.0)
                out.append(dict(J=J, rgb=rgb, residual=res))
            else:
                out.append(dict(rgb=a.numpy(), depth=b.numpy()))
        self.outputs = None
        return out


class Server:
    """Continuous batching over one device-resident map (see module docs)."""

    def __init__(self, gmap: GaussianMap, mem_budget: int = 4 << 30, max_views: int = 8, n_streams: int = 4,
                 use_graphs: bool = True, pairs_per_pixel: float = 4.0, device="cuda", max_bypass: float = 0.02):
        self.gmap, self.mem_budget, self.max_views = gmap, int(mem_budget), int(max_views)
        self.use_graphs = use_graphs
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.pairs_per_pixel = float(pairs_per_pixel)
        self.max_bypass = float(max_bypass)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.runners: dict = collections.defaultdict(list)
        self.waiting: dict = collections.defaultdict(collections.deque)
        self.inbox: queue.Queue = queue.Queue()
        self.inflight = []          # (runner, reqs)
        self.inflight_bytes = 0
        self.max_inflight_bytes = 0
        self._stop = threading.Event()
        self._thread = None
        self._stream_rr = 0
        self.batches = 0
        self.retries = 0
        self.pairs_per_view: dict = {}  # key -> largest pair count one view needed so far
        self.pairs_sum: dict = collections.defaultdict(float)  # key -> (sum of per-view pair counts, views)
        self.pairs_views: dict = collections.defaultdict(int)
        self.runners_added = 0  # runners created while serving (all others came from warmup)
        self.added_keys = []    # (kind, W, H, slots) of those
        self.grows = 0          # workspaces re-allocated for a larger pair demand
        self._build_q: queue.Queue = queue.Queue()
        self._built: queue.Queue = queue.Queue()
        self._building = set()
        self._builder = None

    # ---------------------------------------------------------------- setup
    def _capacity(self, key, slots, headroom: float = 1.25):
        """Pair capacity of a runner: ``headroom`` x the largest per-view demand
        seen, and for several slots at least ``headroom`` x 1.25 x slots x the
        mean demand (several views rarely all need the maximum; an overflow
        re-runs)."""
        _, W, H, _ = key
        if key not in self.pairs_per_view:
            return max(1 << 16, int(self.pairs_per_pixel * W * H * slots))
        mean = self.pairs_sum[key] / max(1, self.pairs_views[key])
        cap = headroom * max(self.pairs_per_view[key], 1.25 * slots * mean)
        return max(1 << 16, int(cap))

    def _observe(self, key, per_view_pairs: int, views: int = 1):
        self.pairs_per_view[key] = max(self.pairs_per_view.get(key, 0), int(per_view_pairs))
        self.pairs_sum[key] += float(per_view_pairs) * views
        self.pairs_views[key] += views

    def calibrate(self, requests):
        """Measure the pair demand of sample requests (one eager, checked
        render each) so that runners are sized before serving starts."""
        rasts = {}
        for r in requests:
            kind, W, H, _ = r.key
            rast = rasts.get((W, H))
            if rast is None:
                rast = rasts[(W, H)] = Rasterizer(self.gmap.n, 1, W, H, pair_capacity=1 << 22, device=self.device)
            rast.project_and_sort(self.gmap, cameras_tensor([r.camera], device=self.device), check=True)
            self._observe(r.key, rast.status()[1])
        del rasts
        torch.cuda.synchronize(self.device)

    def _runner(self, key, slots):
        """A free runner for (key, slots), creating (and capturing) one if none is free."""
        for r in self.runners[(key, slots)]:
            if not r.busy:
                return r
        r = _Runner(self, key, slots, self._capacity(key, slots, headroom=1.6))
        if self.use_graphs:
            # a first eager run only matters before any kernel has been launched
            r.capture(warm=self._thread is None)
        self.runners[(key, slots)].append(r)
        if self._thread is not None:
            self.runners_added += 1
            self.added_keys.append((key[0], key[1], key[2], slots))
        return r

    def _request_build(self, key, slots):
        if (key, slots) not in self._building:
            self._building.add((key, slots))
            self._build_q.put((key, slots, self._capacity(key, slots, headroom=1.6)))

    def _build_loop(self):
        torch.cuda.set_device(self.device)
        while True:
            item = self._build_q.get()
            if item is None:
                return
            key, slots, cap = item
            try:
                r = _Runner(self, key, slots, cap)
                if self.use_graphs:
                    r.capture(warm=False)
                self._built.put(r)
            except BaseException as exc:  # handed to the scheduler, which fails the waiting requests
                self._built.put(exc)

    def _take_built(self):
        while True:
            try:
                r = self._built.get_nowait()
            except queue.Empty:
                return
            if isinstance(r, BaseException):
                raise r
            self.runners[(r.key, r.slots)].append(r)
            self._building.discard((r.key, r.slots))
            self.runners_added += 1
            self.added_keys.append((r.key[0], r.key[1], r.key[2], r.slots))

    def warmup(self, keys, copies: int = 3, pinned_per_key: int = 32):
        """Create and capture runners per (key, slot count) before serving
        (``copies`` of each, two more for single-request batches, which
        overlap most), so that overlapping batches rarely need a new one."""
        for key in keys:
            for s in _slot_counts(self.max_views):
                made = []
                for _ in range(copies + 2 * (s == 1)):
                    r = self._runner(key, s)
                    r.busy = True  # so that the next call makes another
                    made.append(r)
                for r in made:
                    r.busy = False
        # each request's results go to the caller in pinned host tensors from
        # torch's pinned-memory cache; fill the cache now (a pinned allocation
        # of megabytes takes milliseconds) so that requests do not pay for it
        for key in keys:
            kind, W, H, npix = key
            shapes = [(npix, 3, 6), (npix, 3)] if kind == "jacobian" else [(3, H, W), (H, W)]
            held = [torch.empty(sh, pin_memory=True) for _ in range(pinned_per_key) for sh in shapes]
            del held
        torch.cuda.synchronize(self.device)

    # ---------------------------------------------------------------- API
    def submit(self, req: Request) -> Future:
        req.arrival = time.perf_counter()
        self.inbox.put(req)
        return req.future

    def start(self, prime=None):
        """Start the scheduler.  ``prime``: sample requests, one batch of each
        distinct key of which runs on the scheduler thread before it accepts
        work (first launches from a thread pay one-time costs); their results
        are dropped."""
        self._prime = list(prime or [])
        self._ready = threading.Event()
        self._builder = threading.Thread(target=self._build_loop, daemon=True)
        self._builder.start()
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()
        self._ready.wait()

    def stop(self):
        self._stop.set()
        if self._thread is not None:
            self._thread.join()
        if self._builder is not None:
            self._build_q.put(None)
            self._builder.join()

    # ---------------------------------------------------------------- loop
    def _loop(self):
        try:
            torch.cuda.set_device(self.device)
            seen = set()
            for r in self._prime:
                if r.key in seen:
                    continue
                seen.add(r.key)
                for stream in self.streams:
                    runner = self._free_runner(r.key, 1) or self._runner(r.key, 1)
                    runner.launch([r], stream)
                    runner.event.synchronize()
                    runner.outputs = None
            self._ready.set()
            self._run()
        except BaseException as exc:  # never leave callers waiting on a dead loop
            self._ready.set()
            pending = [r for _, rs in self.inflight for r in rs] + [r for q in self.waiting.values() for r in q]
            while not self.inbox.empty():
                pending.append(self.inbox.get_nowait())
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(exc)
            raise

    def _run(self):
        torch.cuda.set_device(self.device)
        while not self._stop.is_set() or self.inflight or any(self.waiting.values()) or not self.inbox.empty():
            self._drain_inbox()
            self._take_built()
            self._complete()
            launched = self._schedule()
            if not launched and not self.inflight:
                try:
                    req = self.inbox.get(timeout=0.001)
                    self.waiting[req.key].append(req)
                except queue.Empty:
                    pass
            elif not launched:
                time.sleep(5e-5)  # batches in flight: poll their events without holding a core

    def _drain_inbox(self):
        while True:
            try:
                req = self.inbox.get_nowait()
            except queue.Empty:
                return
            self.waiting[req.key].append(req)

    def _free_runner(self, key, slots):
        for r in self.runners[(key, slots)]:
            if not r.busy:
                return r
        return None

    def _admit(self, key, n):
        """(runner, requests to take) for up to ``n`` waiting requests of
        ``key``: the smallest slot count that holds all of them if its sort
        buffers fit in the free budget, else the largest smaller one that fits;
        anything runs when nothing else is in flight."""
        free = self.mem_budget - self.inflight_bytes
        counts = _slot_counts(self.max_views)
        order = [s for s in counts if s >= n][:1] + [s for s in reversed(counts) if s < n]
        for slots in order:
            runner = self._free_runner(key, slots)
            target = self._capacity(key, slots, headroom=1.6)
            need = SORT_BYTES_PER_PAIR * (target if runner is None or
                                          runner.rast.capacity < self._capacity(key, slots, headroom=1.0)
                                          else runner.rast.capacity)
            if need > free and self.inflight:
                continue
            if runner is None:
                if self.inflight:
                    # built on the builder thread; meanwhile smaller batches, or wait for a free runner
                    self._request_build(key, slots)
                    continue
                runner = self._runner(key, slots)
            elif runner.rast.capacity < self._capacity(key, slots, headroom=1.0):
                # the pair demand seen for this key outgrew the runner: grow it
                # before use, with room for further growth of the estimate
                runner.grow(target)
                self.grows += 1
            return runner, min(n, slots)
        return None

    def _schedule(self) -> bool:
        launched = False
        now = time.perf_counter()
        # oldest waiting request first; a key whose batch does not fit the free
        # budget lets later keys use it until its oldest request has waited
        # max_bypass seconds, then everything waits for it
        keys = sorted((k for k, q in self.waiting.items() if q), key=lambda k: self.waiting[k][0].arrival)
        for key in keys:
            q = self.waiting[key]
            while q:
                pick = self._admit(key, min(len(q), self.max_views))
                if pick is None:
                    if now - q[0].arrival > self.max_bypass:
                        return launched
                    break
                runner, n = pick
                reqs = [q.popleft() for _ in range(n)]
                t_launch = time.perf_counter()
                for r in reqs:
                    r.launched = t_launch
                runner.busy = True
                stream = self.streams[self._stream_rr % len(self.streams)]
                self._stream_rr += 1
                if self.use_graphs and runner.graph is None:
                    runner.capture(warm=False)
                runner.launch(reqs, stream)
                runner.bytes_launched = runner.bytes
                self.inflight.append((runner, reqs))
                self.inflight_bytes += runner.bytes
                self.max_inflight_bytes = max(self.max_inflight_bytes, self.inflight_bytes)
                self.batches += 1
                launched = True
        return launched

    def _complete(self):
        still = []
        for runner, reqs in self.inflight:
            if not runner.event.query():
                still.append((runner, reqs))
                continue
            key = reqs[0].key
            needed = int(runner.host_status[1])
            self._observe(key, -(-needed // runner.slots), len(reqs))
            if int(runner.host_status[0]) != 0:
                # pair buffer overflow: grow the runner (re-captured before its
                # next launch) and put the requests back at the head of their queue
                self.retries += 1
                runner.grow(int(1.25 * needed) + 1024)
                runner.outputs = None
                runner.busy = False
                self.inflight_bytes -= runner.bytes_launched
                self.waiting[key].extendleft(reversed(reqs))
                continue
            t = time.perf_counter()
            for r, res in zip(reqs, runner.results(reqs)):
                r.done = t
                if r.on_result is not None:
                    r.on_result(r, res)
                    res = None
                r.future.set_result(res)
            runner.busy = False
            self.inflight_bytes -= runner.bytes_launched
        self.inflight = still


class PlainRenderer:
    """One request at a time, one launch sequence per request, no graphs: the
    reference point for the server.

    By default (``checked=False``) a request runs the way the server runs a
    batch, minus the batching and the graphs: the camera (and pixel list) go
    up from pinned host memory, nothing is read back between sort and blend,
    the results are copied asynchronously into pinned host tensors, and the
    status is read once, when the request's work has finished (a pair-buffer
    overflow is then retried with a larger buffer).  ``checked=True`` is the
    simplest plain loop: the status is read back after the sort (a full
    synchronisation before the blend) and results come back with ``.cpu()``
    (pageable copies)."""

    def __init__(self, gmap: GaussianMap, device="cuda", checked: bool = False):
        self.gmap = gmap
        self.device = torch.device(device)
        self.checked = bool(checked)
        self.rasts = {}
        self.outs = {}
        self.retries = 0
        self.cams = torch.zeros(1, 16, device=self.device)
        self.host_cams = torch.empty(1, 16, pin_memory=True)
        self.status = torch.zeros(2, dtype=torch.int32, device=self.device)
        self.host_status = torch.zeros(2, dtype=torch.int32, pin_memory=True)
        self.event = torch.cuda.Event()
        self.pix = {}

    def _setup(self, req):
        kind, W, H, npix = req.key
        key = (W, H)
        if key not in self.rasts:
            self.rasts[key] = Rasterizer(self.gmap.n, 1, W, H, device=self.device)
            f = dict(device=self.device, dtype=torch.float32)
            self.outs[key] = RenderOut(torch.empty(1, 3, H, W, **f), torch.empty(1, H, W, **f),
                                       torch.empty(1, H, W, **f), torch.empty(1, H, W, **f),
                                       torch.empty(1, H, W, dtype=torch.int32, device=self.device))
        return kind, key, self.rasts[key]

    def run(self, req: Request):
        kind, key, rast = self._setup(req)
        if self.checked:
            cams = cameras_tensor([req.camera], device=self.device)
            out = rast.render(self.gmap, cams, check=True)
            if kind == "jacobian":
                pix = torch.as_tensor(req.pix, device=self.device).view(1, -1)
                J, rgb = rast.pose_jacobian(self.gmap, cams, pix)
                J, rgb = J[0].cpu().numpy(), rgb[0].cpu().numpy()
                return dict(J=J, rgb=rgb, residual=rgb - (req.target if req.target is not None else 0.0))
            return dict(rgb=out.rgb[0].cpu().numpy(), depth=out.depth[0].cpu().numpy())
        self.host_cams[0] = torch.as_tensor(cameras_tensor([req.camera], device="cpu")[0])
        self.cams.copy_(self.host_cams, non_blocking=True)
        if kind == "jacobian":
            npix = len(req.pix)
            if npix not in self.pix:
                self.pix[npix] = (torch.zeros(1, npix, dtype=torch.int32, device=self.device),
                                  torch.empty(1, npix, dtype=torch.int32, pin_memory=True))
            pix, host_pix = self.pix[npix]
            host_pix[0] = torch.as_tensor(req.pix)
            pix.copy_(host_pix, non_blocking=True)
        out = self.outs[key]
        while True:
            rast.render(self.gmap, self.cams, check=False, out=out)
            if kind == "jacobian":
                J, jrgb = rast.pose_jacobian(self.gmap, self.cams, pix)
                a = torch.empty(J.shape[1:], pin_memory=True)
                b = torch.empty(jrgb.shape[1:], pin_memory=True)
                a.copy_(J[0], non_blocking=True)
                b.copy_(jrgb[0], non_blocking=True)
            else:
                a = torch.empty(out.rgb.shape[1:], pin_memory=True)
                b = torch.empty(out.depth.shape[1:], pin_memory=True)
                a.copy_(out.rgb[0], non_blocking=True)
                b.copy_(out.depth[0], non_blocking=True)
            self.status.copy_(rast._view(rast.layout.counters, 2, torch.int32))
            self.host_status.copy_(self.status, non_blocking=True)
            self.event.record()
            self.event.synchronize()
            code, needed = int(self.host_status[0]), int(self.host_status[1])
            if code == N.GS_OK:
                break
            if code != N.GS_ERR_CAPACITY:
                raise N.GsError("plain render", code)
            self.retries += 1
            rast.capacity = int(1.25 * needed) + 1024
            rast._alloc()
        if kind == "jacobian":
            rgb = b.numpy()
            return dict(J=a.numpy(), rgb=rgb, residual=rgb - (req.target if req.target is not None else 0.0))
        return dict(rgb=a.numpy(), depth=b.numpy())


def latency_stats(reqs):
    """p50/p99/mean of arrival -> result latency; for server requests also the
    queueing part (arrival -> batch launch)."""
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    out = dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
               mean_ms=float(lat.mean()), n=len(lat))
    if all(r.launched for r in reqs):
        wait = np.array([r.launched - r.arrival for r in reqs]) * 1e3
        out.update(queue_p50_ms=float(np.percentile(wait, 50)), queue_p99_ms=float(np.percentile(wait, 99)))
    return out
