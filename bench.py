#!/usr/bin/env python3
"""Benchmark of the differentiable 3DGS rasterizer (Gaussian-LIC2 mapping step).

Workload: 1,000,000 Gaussians in a 60x20x60 m box (SH degree 3, FP32), a
batch of 4 keyframes at 1920x1080 (fx = fy = 1000) on a straight track, each
with a smooth random target image and a 32-ring LiDAR sparse depth map; loss
0.8 L1 colour + 0.2 opacity-normalised L1 depth.  One step = projection and
tile culling, binning and sort, forward compositing, fused loss backward to
every Gaussian parameter and to the 4 camera poses.  Metric: fwd+bwd Mpix/s
(4 x 1920 x 1080 pixels per step).

``python bench.py [--gpus N] [--steps K] [--warmup W]`` prints one JSON line;
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload instead.  N > 1 runs under torchrun as independent replicas
(one batch of keyframes per GPU, no collective on the data path).
"""
from __future__ import annotations

import argparse
import csv
import datetime as dt
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="mapping fwd+bwd, 1M Gaussians SH3 FP32, 4 keyframes 1920x1080", n_gaussians=1_000_000,
                sh_degree=3, views=4, width=1920, height=1080, focal=1000.0, loss="0.8 L1 rgb + 0.2 L1 depth/opacity")
METRIC = "fwd+bwd Mpix/s at 1M Gaussians"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=WORKLOAD["n_gaussians"])
    p.add_argument("--views", type=int, default=WORKLOAD["views"], help="keyframes per batch (profiling runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    p.add_argument("--no-bucket", action="store_true", help="skip the per-Gaussian (bucket) backward leg")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="target length of the CPU baseline sample")
    p.add_argument("--cpu-seconds-one-core", type=float, default=4.0,
                   help="length of the one-core oracle sample beside the CPU baseline (0 skips it)")
    p.add_argument("--reference-seconds", type=float, default=150.0,
                   help="--impl reference: oracle time spread over the warm-up and timed steps")
    p.add_argument("--tracking-frames", type=int, default=32,
                   help="frames in the tracking measurement (0 skips it): 1M Gaussians SH1, 640x512, N_t = 30")
    p.add_argument("--serving-requests", type=int, default=10000,
                   help="requests in the serving measurement (0 skips it): the serving workload's 10,000")
    return p.parse_args()


# ----------------------------------------------------------------- ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    def __init__(self, use_cuda: bool):
        import torch
        import torch.distributed as td
        self.rank, self.world, self.local = dist_env()
        self.td = td if self.world > 1 else None
        self.torch = torch
        self.dev = torch.device("cuda", self.local) if use_cuda else torch.device("cpu")
        if self.td is not None:
            backend = "nccl" if use_cuda else "gloo"
            kw = dict(device_id=self.dev) if use_cuda else {}
            td.init_process_group(backend, **kw)

    def barrier(self):
        if self.td is not None:
            self.td.barrier()

    def max(self, x: float) -> float:
        if self.td is None:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.dev)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.td is None:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.dev)
        self.td.all_reduce(t, op=self.td.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.td is not None:
            self.td.destroy_process_group()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling (every 50 ms) of SM clocks and throttle reasons."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = list(csv.reader(io.StringIO(open(self.tmp.name).read())))
        os.unlink(self.tmp.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside, allr = [], []
        for r in rows:
            if len(r) < 10:
                continue
            try:
                ts = dt.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rec = dict(ts=ts, sm=float(r[2]), smax=float(r[3]),
                           flags={n: r[6 + i].strip() == "Active" for i, n in enumerate(names)})
            except ValueError:
                continue
            allr.append(rec)
            if t0 - 0.05 <= rec["ts"] <= t1 + 0.05:
                inside.append(rec)
        use = inside if inside else allr
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = sorted({n for rec in use for n, on in rec["flags"].items() if on})
        return {"sm_mhz": statistics.median(r["sm"] for r in use), "sm_max_mhz": max(r["smax"] for r in use),
                "reasons": reasons, "samples": len(use), "window": "timed region" if inside else "whole run"}


# ----------------------------------------------------------------- helpers
def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0, "source": "fallback"}


def source_hash(*names) -> str:
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2507_04004_b300", "csrc", n), "rb").read())
    h.update(open(os.path.join(ROOT, "paper_2507_04004_b300", "csrc", "gs_device.cuh"), "rb").read())
    return h.hexdigest()[:16]


# Which source file holds each kernel (for matching ncu traffic to source).
KERNEL_SRC = {"project": "project.cu", "scan_buckets": "binning.cu", "depth_hist": "binning.cu",
              "depth_scan": "binning.cu", "depth_scatter": "binning.cu", "entry_order": "binning.cu",
              "entry_units": "binning.cu", "entry_rows": "binning.cu", "unit_scan": "binning.cu",
              "scatter_rows": "binning.cu", "rows_count": "binning.cu", "scan": "binning.cu",
              "rows_emit": "binning.cu", "render_fwd": "render_fwd.cu", "count_depth": "render_bwd.cu",
              "render_bwd": "render_bwd.cu", "preprocess_bwd": "render_bwd.cu", "pose_jacobian": "jacobian.cu",
              "tile_work": "render_bwd.cu"}


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel's source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d or d.get("source_hash") != source_hash(KERNEL_SRC[kernel]):
        return None
    return d.get("bytes_per_launch_full_workload")


def make_workload(n: int, seed_offset: int = 0, views: int = WORKLOAD["views"]):
    from paper_2507_04004_b300 import synth
    return synth.mapping(seed=synth.SEED_BASE + 20 + seed_offset, n=n, width=WORKLOAD["width"],
                         height=WORKLOAD["height"], focal=WORKLOAD["focal"], sh_degree=WORKLOAD["sh_degree"],
                         n_views=views)


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(w, seconds_budget: float, calibrate: dict | None = None):
    """Time the FP64 oracle's fwd+bwd over a centred pixel rectangle of view 0
    sized to take about ``seconds_budget``; returns (pixels, seconds, rect)."""
    from oracle import oracle as O
    W, H = w.cams[0]["width"], w.cams[0]["height"]
    m = w.gmap.as_dict()
    cal = calibrate if calibrate is not None else {}
    if "per_px" not in cal:
        side = 128
        rect = (W // 2 - side // 2, H // 2 - side // 2, side, side)
        t0 = time.perf_counter()
        O.backward(m, w.cams[:1], tgt_rgb=w.tgt_rgb[:1], tgt_depth=w.tgt_depth[:1], w_rgb=w.w_rgb,
                   w_depth=w.w_depth, rect=rect)
        t = time.perf_counter() - t0
        cal["fixed"] = 0.7 * t
        cal["per_px"] = max(t * 0.3 / (side * side), 1e-8)
    area = max(64 * 64, (seconds_budget - cal["fixed"]) / cal["per_px"])
    if area >= W * H:
        rect = (0, 0, W, H)
    else:
        side = int(area ** 0.5)
        rw, rh = min(W, int(side * 16 / 9)), min(H, int(side * 9 / 16))
        rw, rh = max(64, rw), max(64, rh)
        rect = ((W - rw) // 2, (H - rh) // 2, rw, rh)
    t0 = time.perf_counter()
    O.backward(m, w.cams[:1], tgt_rgb=w.tgt_rgb[:1], tgt_depth=w.tgt_depth[:1], w_rgb=w.w_rgb, w_depth=w.w_depth,
               rect=rect)
    t = time.perf_counter() - t0
    return rect[2] * rect[3], t, rect


def oracle_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    w = make_workload(args.n)
    budget = max(0.5, args.reference_seconds / max(1, args.steps + args.warmup))
    cal = {}
    for _ in range(args.warmup):
        oracle_sample(w, budget, cal)
    pix, secs = 0, 0.0
    rect = None
    for _ in range(args.steps):
        p, t, rect = oracle_sample(w, budget, cal)
        pix += p
        secs += t
    value = pix / secs / 1e6
    sample = f"view 0 of the workload, centred {rect[2]}x{rect[3]} pixel rectangle per step, fwd+bwd in FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="oracle on host cores"),
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(args, d, rast, gm, w, px_step):
    """Same metric through the public API from host buffers: every step
    uploads its keyframes (8-bit images, LiDAR depth pairs, cameras) from
    pinned memory on a copy stream (double-buffered), expands the depth pairs
    as the first work of its graph on the compute stream, and reads the loss
    back."""
    import torch

    from paper_2507_04004_b300 import synth
    from paper_2507_04004_b300.pipeline import HostKeyframes, MappingStep
    from paper_2507_04004_b300.raster import cameras_tensor
    kf = HostKeyframes.from_dense(synth.to_uint8(w.tgt_rgb), w.tgt_depth, cameras_tensor(w.cams, device="cpu"))
    ms_step = MappingStep(rast, gm, w.w_rgb, w.w_depth)
    e_steps = max(10, min(args.steps, 50))
    slot = ms_step.upload(kf)
    for _ in range(3):
        nxt = ms_step.upload(kf)
        ms_step.step(slot)
        slot = nxt
    torch.cuda.synchronize()
    d.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    slot = ms_step.upload(kf)
    for i in range(e_steps):
        nxt = ms_step.upload(kf) if i + 1 < e_steps else None
        ms_step.step(slot)
        slot = nxt
    e1.record()
    torch.cuda.synchronize()
    e2e_s = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
    e2e_s = d.max(e2e_s)
    d.barrier()
    val = d.sum(px_step * e_steps) / e2e_s / 1e6
    return {"value": round(val, 2), "unit": "Mpix/s", "h2d_bytes_per_step": ms_step.h2d_bytes,
            "d2h_bytes_per_step": ms_step.d2h_bytes}


def serving_workload(n_requests: int, seed: int = 2507_04004 + 5, n_calib: int = 64):
    """3M-Gaussian map (SH 3, BF16), requests: 70 % renders at 640x360,
    1280x720 or 1920x1080 (focal 0.52 W) and 30 % tracking-Jacobian requests at
    640x512 with the 20k highest-gradient pixels, random poses inside the map,
    Poisson arrivals at 200 requests/s; plus ``n_calib`` further requests from
    the same distribution for sizing the server's buffers (not measured)."""
    import numpy as np

    from paper_2507_04004_b300 import synth
    from paper_2507_04004_b300.serve import Request
    rng = np.random.default_rng(seed)
    lo, hi = (-30.0, -10.0, -30.0), (30.0, 10.0, 30.0)
    g = synth.random_map(rng, 3_000_000, lo, hi, 3)
    pool = []
    for _ in range(4):  # a few tracking targets / pixel selections, reused
        img = synth.smooth_target(rng, 512, 640)
        pix = synth.top_gradient_pixels(img, 20_000)
        pool.append((pix, img.reshape(3, -1)[:, pix].T.copy()))
    sizes = [(640, 360), (1280, 720), (1920, 1080)]
    reqs = []
    for i, (centre, Rc) in enumerate(synth.tracking_poses(rng, n_requests + n_calib, lo, hi)):
        R, t = synth.pose_from_centre(Rc, centre)
        if rng.random() < 0.3:
            pix, tgt = pool[i % len(pool)]
            reqs.append(Request("jacobian", synth.camera(R, t, 500.0, 500.0, 320, 256, 640, 512), pix=pix, target=tgt))
        else:
            W, H = sizes[int(rng.integers(0, 3))]
            reqs.append(Request("render", synth.camera(R, t, 0.52 * W, 0.52 * W, W / 2, H / 2, W, H)))
    gaps = rng.exponential(1.0 / 200.0, n_requests)
    return g, reqs[:n_requests], np.cumsum(gaps), reqs[n_requests:]


def run_mapping_iteration(args, rast, gm, cams, w, tgt_rgb, tgt_depth):
    """The paper's full mapping iteration on the bench workload (Eq.
    depth_loss with its D-SSIM term): render, L = 0.8 L1 + 0.2 D-SSIM
    + 0.005 L_depth, backward, sparse Adam (which also clears the gradients it
    used, so no whole-map clear).  Timed after the headline measurement; the
    map is changed by the optimiser."""
    import torch

    from paper_2507_04004_b300.raster import DSSIM, SparseAdam
    V, H, W = args.views, WORKLOAD["height"], WORKLOAD["width"]
    dssim = DSSIM(V, H, W, device=gm.mean.device)
    opt = SparseAdam(gm)
    out = rast.render(gm, cams, check=False)
    grads = rast.new_grads(gm)
    dl = torch.zeros_like(out.rgb)

    def it():
        rast.render(gm, cams, check=False, out=out)
        dl.zero_()
        dssim(out.rgb, tgt_rgb, 0.2, loss=grads.loss, dl_dimg=dl)
        rast.backward(gm, cams, out, tgt_rgb=tgt_rgb, tgt_depth=tgt_depth, w_rgb=0.8, w_depth=0.005, dl_drgb=dl,
                      grads=grads)
        opt.step(gm, grads, rast)

    for _ in range(5):
        it()
    torch.cuda.synchronize()
    n = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        it()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    code, _ = rast.status()
    if code != 0:
        raise SystemExit(f"workspace status {code} in the mapping-iteration leg")
    return {"loss": "0.8 L1 + 0.2 D-SSIM + 0.005 L_depth (Eq. depth_loss), sparse Adam (3DGS learning rates)",
            "ms_per_iteration": round(ms, 4), "mpix_per_s": round(V * H * W / (ms / 1e3) / 1e6, 1)}


# Algorithmic lane operations per (pixel, list position) evaluation of the
# blend kernels, as the method computes it (one per scalar operation, an FMA
# counts one; per-column terms shared by a thread's pixels amortised), for a
# blended evaluation and one skipped below alpha_min; then the same in FP32
# FLOP with an FMA counted twice.
#   forward, skipped: power 3 (dy, two FMA) + column terms 1 + alpha_min test 1 = 5
#   forward, blended: + ex2 1, clamp 1, 1 - alpha 1, T (1 - alpha) 1, stop test 1,
#                     w = alpha T 1, colour and depth 4, last index 1 = 16
#   backward, skipped: 5 (as forward)
#   backward, blended: + ex2 1, clamp 1, 1 - alpha 1, T recovery (reciprocal, product) 2,
#                      w 1, adjoint dot (gC.c + gD d + gO) 4, minus behind-sum 1, dL/dalpha 1,
#                      behind-sum update 1, dL/dc and dL/dd sums 4, dL/dpower 1, moment sums 3,
#                      per-thread moment finish 1.5 (12 per 8 pixels) = 28.5
BLEND_OPS = {  # kernel: (blended ops, skipped ops, blended FLOP, skipped FLOP)
    "render_fwd": (16.0, 5.0, 23.0, 8.0),
    "render_bwd": (28.5, 5.0, 45.0, 8.0),
}


def step_model(n, views, hw, n_vis, n_rows, n_pairs, n_listed, p_proc, k_blend, k_skip, k_tested=None,
               sh_degree=None):
    """Algorithmic (bytes, lane operations) per launch of every kernel of the
    mapping step, from the step's work counters.  Bytes: what the method must
    move to or from HBM at least once; operations: the arithmetic the method
    performs (see BLEND_OPS for the blend kernels).
      project:  44 B parameters per Gaussian + SH per visible entry + 100 B
                written per visible entry (48 record, 48 cleared adjoint,
                4 list) + 8 B tile box per (view, Gaussian); ~300 ops per
                visible entry (rotation, covariance, Jacobian, conic, SH 3,
                box), 40 per (view, Gaussian) for the near/screen test
      depth sort: depth_hist reads 8 B per visible entry once (digit counts
                of all passes); depth_scatter (5 passes at 2..256 views)
                reads 8 B and writes 8 B per entry per pass; ~12 ops per
                entry per pass
      entry_order: 8 B read, 4 B written per visible entry
      entry_rows / scatter_rows: per visible entry 4 B list + 8 B box
                read (twice), 4 B row item written per row item
      rows_count: per row item 4 B item + 32 B record read, 4 B span
                written; 16 chords x 14 ops
      rows_emit: per row item 4 + 4 B read, 4 B Gaussian index written per
                pair; ~10 ops per pair
      render_fwd: 52 B (record + index) per processed pair, 28 B per pixel
                written (RGB, depth, opacity, T_final, n_contrib); operations
                per blended evaluation and per other list position a pixel
                tests (up to the Gaussian it stops at, else its tile's whole
                list: positions past the last contributor still need the test)
      render_bwd: 44 B per pixel read (RGB, target RGB, depth, opacity,
                T_final, n_contrib, target depth), 52 B per processed pair,
                48 B of 2D adjoints added per processed pair
      preprocess_bwd: per listed Gaussian parameters + SH read and their
                gradients read and written ((44 + SH) x 3); per visible
                entry 96 B (record, adjoint); ~300 ops per visible entry
      count_depth: 4 B per pixel.
      tile_work: n_contrib read (4 B per pixel), per (view, tile) item its
                class slot taken and written; a max per pixel, ~40 ops per
                item."""
    deg = WORKLOAD["sh_degree"] if sh_degree is None else sh_degree
    b_sh = 4 * 3 * (deg + 1) ** 2
    px = views * hw
    k_fwd = k_tested if k_tested is not None else k_blend + k_skip  # evaluations the forward makes
    tiles = views * ((WORKLOAD["width"] + 15) // 16) * ((WORKLOAD["height"] + 15) // 16)
    passes = 4 + (1 if views > 1 else 0)
    return {
        "project": (44.0 * n + b_sh * n_vis + 100.0 * n_vis + 8.0 * views * n + 8.0 * n_vis,
                    300.0 * n_vis + 40.0 * views * n),
        "depth_hist": (8.0 * n_vis, 4.0 * n_vis * passes),
        "depth_scatter": (16.0 * n_vis * passes, 12.0 * n_vis * passes),
        "entry_order": (12.0 * n_vis, 8.0 * n_vis),
        "entry_rows": (12.0 * n_vis, 6.0 * n_vis),
        "scatter_rows": (12.0 * n_vis + 4.0 * n_rows, 10.0 * n_rows),
        "rows_count": (40.0 * n_rows, 16 * 14.0 * n_rows),
        "rows_emit": (8.0 * n_rows + 4.0 * n_pairs, 10.0 * n_pairs),
        "render_fwd": (52.0 * p_proc + 28.0 * px,
                       k_blend * BLEND_OPS["render_fwd"][0] + (k_fwd - k_blend) * BLEND_OPS["render_fwd"][1]),
        "count_depth": (4.0 * px, 2.0 * px),
        "tile_work": (4.0 * px + 8.0 * tiles, 2.0 * px + 40.0 * tiles),
        "render_bwd": (44.0 * px + 100.0 * p_proc,
                       k_blend * BLEND_OPS["render_bwd"][0] + k_skip * BLEND_OPS["render_bwd"][1]),
        "preprocess_bwd": ((44.0 + b_sh) * 3 * n_listed + 96.0 * n_vis, 300.0 * n_vis),
    }


def tile_max_prefix(n_contrib) -> int:
    """Pairs the blend kernels process: per 16x16 tile the longest
    contributor prefix of its pixels, summed over tiles and views."""
    import torch.nn.functional as F
    V, H, W = n_contrib.shape
    x = n_contrib.float().view(V, 1, H, W)  # counts far below 2^24: exact in FP32
    x = F.pad(x, (0, (-W) % 16, 0, (-H) % 16))
    return int(F.max_pool2d(x, 16).sum().item())


def run_bucket_backward(args, rast0, gm, cams, tgt_rgb, tgt_depth, w, k_blend, k_skip, issue):
    """The headline step with the per-Gaussian (bucket) blend backward of
    Sec. "Per-Gaussian Backpropagation" in place of the pixel-parallel one
    (the forward then writes its bucket checkpoints): throughput and
    per-kernel times on the same map, cameras and targets."""
    import numpy as np
    import torch

    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import Rasterizer
    V, H, W = args.views, WORKLOAD["height"], WORKLOAD["width"]
    rast = Rasterizer(gm.n, V, W, H, pair_capacity=rast0.capacity, device=gm.mean.device, backward="bucket")
    out = rast.render(gm, cams, check=True)
    grads = rast.new_grads(gm)

    def step():
        grads.zero_()
        rast.render(gm, cams, check=False, out=out)
        rast.backward(gm, cams, out, tgt_rgb=tgt_rgb, tgt_depth=tgt_depth, w_rgb=w.w_rgb, w_depth=w.w_depth,
                      grads=grads)

    for _ in range(5):
        step()
    torch.cuda.synchronize()
    n = 30
    cap = 20 * n + 16
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * cap)]
    for e in evs:
        e.record()
    ids = np.zeros(cap, np.int32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    N.gs_trace_start([e.cuda_event for e in evs], ids)
    e0.record()
    for _ in range(n):
        step()
    e1.record()
    e1.synchronize()
    launches = N.gs_trace_stop()
    torch.cuda.synchronize()
    code, _ = rast.status()
    if code != 0:
        raise SystemExit(f"workspace status {code} in the bucket-backward leg")
    ms = e0.elapsed_time(e1) / n
    per = {}
    for k in range(min(launches, cap)):
        a = per.setdefault(N.gs_kernel_name(int(ids[k])), [0, 0.0])
        a[0] += 1
        a[1] += evs[2 * k].elapsed_time(evs[2 * k + 1])
    kern = {k: round(v[1] / v[0], 4) for k, v in sorted(per.items(), key=lambda x: -x[1][1])}
    bwd_ms = kern.get("render_bwd_bucket", 0.0)
    res = {"ms_per_step": round(ms, 4), "mpix_per_s": round(V * H * W / (ms / 1e3) / 1e6, 1), "kernels_ms": kern,
           # the same algorithmic instruction count as the pixel-parallel backward, against instruction issue
           "blend_bwd_issue_frac": round((k_blend * BLEND_OPS["render_bwd"][0] + k_skip * BLEND_OPS["render_bwd"][1])
                                         / 32.0 / (bwd_ms / 1e3) / issue, 4) if bwd_ms else None,
           "bucket_workspace_bytes": int(rast._bucket_buf.numel())}
    del rast, out, grads
    torch.cuda.empty_cache()
    return res


def run_tracking(args, dev):
    """Pose tracking with the map fixed (N_t = 30 Adam iterations of
    1/2 L1 + 1/2 D-SSIM per frame, all frames as one batch, one captured
    graph): frames per second and the pose error before and after."""
    import numpy as np
    import torch

    from paper_2507_04004_b300 import synth
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    from paper_2507_04004_b300.track import PoseTracker
    V = args.tracking_frames
    w = synth.tracking(n_frames=V)
    gm, _ = GaussianMap.from_host(w.gmap, device=dev).spatially_ordered()  # map build: Morton order
    H, W = 512, 640
    r = Rasterizer(gm.n, V, W, H, device=dev)
    targets = r.render(gm, cameras_tensor(w.meta["gt_cams"], device=dev)).rgb.clone()  # images at the true poses
    del r
    tr = PoseTracker(gm, V, W, H, iters=30, device=dev)
    q = cameras_tensor(w.cams, device=dev)
    for _ in range(2):  # sizing pass, capture, first replay
        xi, loss = tr.track(q, targets)
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        xi, loss = tr.track(q, targets)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # camera factor option 2's residual r = Log(T(t) T~^-1) per frame, with T(t) the poses tracking
    # started from (the trajectory's prediction) and, for reference, the true poses
    res = tr.residual(q).cpu().numpy().astype(np.float64)
    res_gt = tr.residual(cameras_tensor(w.meta["gt_cams"], device=dev)).cpu().numpy().astype(np.float64)
    xi = xi.cpu().numpy().astype(np.float64)
    true = -w.meta["xi"]
    rot0 = np.degrees(np.linalg.norm(true[:, 3:], axis=1))
    rot1 = np.degrees(np.linalg.norm(xi[:, 3:] - true[:, 3:], axis=1))
    tr0 = np.linalg.norm(true[:, :3], axis=1)
    tr1 = np.linalg.norm(xi[:, :3] - true[:, :3], axis=1)
    return {"workload": f"1M Gaussians SH1, {V} frames 640x512 (fx = 500) tracked together, N_t = 30, "
                        "loss 1/2 L1 + 1/2 D-SSIM, start GT Exp(xi) with theta ~ N(0, 0.02 rad), rho ~ N(0, 0.05 m)",
            "ms_per_batch": round(ms, 3), "frames_per_s": round(V / (ms / 1e3), 1),
            "ms_per_iteration": round(ms / 30, 4),
            "rot_err_deg_median": [round(float(np.median(rot0)), 4), round(float(np.median(rot1)), 4)],
            "trans_err_m_median": [round(float(np.median(tr0)), 4), round(float(np.median(tr1)), 4)],
            "residual_log_median": {
                "vs_start_pose": {"rho_m": round(float(np.median(np.linalg.norm(res[:, :3], axis=1))), 4),
                                  "theta_deg": round(float(np.degrees(np.median(np.linalg.norm(res[:, 3:], axis=1)))), 4)},
                "vs_true_pose": {"rho_m": round(float(np.median(np.linalg.norm(res_gt[:, :3], axis=1))), 4),
                                 "theta_deg": round(float(np.degrees(np.median(np.linalg.norm(res_gt[:, 3:], axis=1)))), 4)}},
            "note": "errors [before, after]; timed: the captured 30-iteration graph incl. the status read-back"}


def run_serving(args, dev):
    """p50/p99 latency under Poisson arrivals and closed-loop throughput,
    batched server vs plain one-request-at-a-time rendering."""
    import copy
    import threading

    import torch

    from paper_2507_04004_b300.raster import GaussianMap
    from paper_2507_04004_b300.serve import PlainRenderer, Server, latency_stats
    g, reqs, arrivals, calib = serving_workload(args.serving_requests)
    gm, _ = GaussianMap.from_host(g, device=dev, sh_bf16=True).spatially_ordered()  # map build: Morton order
    def drop(req, res):  # the consumer reads nothing back: results are released at once
        pass

    def fresh():
        out = []
        for r in reqs:
            c = copy.copy(r)
            c.on_result = drop
            out.append(c)
        return out
    out = {"workload": f"3M Gaussians SH3 BF16, {len(reqs)} requests, Poisson 200/s, 70% renders "
                       "(640x360/1280x720/1920x1080), 30% tracking Jacobians (640x512, 20k px)",
           "mem_budget_gib": 4}

    def open_loop(submit_one, rs):
        t0 = time.perf_counter()
        for r, t in zip(rs, arrivals):
            wait = t0 + t - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            submit_one(r)

    # batched server
    srv = Server(gm, mem_budget=4 << 30, max_views=4, n_streams=4, pairs_per_pixel=8.0, device=dev)
    srv.calibrate(calib)
    srv.warmup({r.key for r in reqs})
    srv.start(prime=calib)
    rs = fresh()
    for r in rs:
        r.future = type(r.future)()
    open_loop(lambda r: srv.submit(r), rs)
    for r in rs:
        r.future.result()
    out["server_open_loop"] = latency_stats(rs)
    rs = fresh()
    for r in rs:
        r.future = type(r.future)()
    t0 = time.perf_counter()
    for r in rs:
        srv.submit(r)
    for r in rs:
        r.future.result()
    out["server_req_per_s"] = len(rs) / (time.perf_counter() - t0)
    srv.stop()
    out["server_batches"] = srv.batches
    out["server_retries"] = srv.retries
    out["server_runners_added"] = srv.runners_added
    out["server_runners_added_keys"] = [f"{k} {w}x{h} x{s}" for k, w, h, s in srv.added_keys]
    out["server_grows"] = srv.grows
    out["server_pairs_per_view_max"] = {f"{k[0]} {k[1]}x{k[2]}": v for k, v in srv.pairs_per_view.items()}
    out["server_max_inflight_sort_gib"] = round(srv.max_inflight_bytes / 2 ** 30, 3)
    del srv
    torch.cuda.empty_cache()

    def plain_leg(plain, rs_all, label):
        """The plain path: one worker, FIFO, one launch sequence per request;
        open loop at the same arrival times, then closed loop."""
        for r in reqs[:8]:
            plain.run(r)  # warm-up
        rs = rs_all()
        q, done_all = [], threading.Event()
        lock = threading.Condition()

        def worker():
            k = 0
            while k < len(rs):
                with lock:
                    while len(q) <= k:
                        lock.wait()
                r = q[k]
                plain.run(r)
                r.done = time.perf_counter()
                k += 1
            done_all.set()

        th = threading.Thread(target=worker)
        th.start()

        def submit_plain(r):
            r.arrival = time.perf_counter()
            with lock:
                q.append(r)
                lock.notify()
        open_loop(submit_plain, rs)
        done_all.wait()
        th.join()
        out[f"{label}_open_loop"] = latency_stats(rs)
        rs = rs_all()
        t0 = time.perf_counter()
        for r in rs:
            plain.run(r)
        out[f"{label}_req_per_s"] = len(rs) / (time.perf_counter() - t0)

    # plain path as the server runs a batch (pinned asynchronous copies, one
    # status read per request), then the simplest plain loop (status read
    # back between sort and blend, pageable copies) on the first 2,000 requests
    plain = PlainRenderer(gm, device=dev)
    plain_leg(plain, fresh, "plain")
    out["plain_retries"] = plain.retries
    n_checked = min(len(reqs), 2000)
    plain_leg(PlainRenderer(gm, device=dev, checked=True), lambda: fresh()[:n_checked], "plain_checked")
    out["plain_checked_note"] = (f"first {n_checked} requests; status read back after the sort of every request "
                                 "(a full synchronisation before the blend), results copied with .cpu()")
    out["throughput_ratio"] = out["server_req_per_s"] / out["plain_req_per_s"]
    return out


# ----------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    d = Dist(use_cuda=True)
    torch.cuda.set_device(d.dev)
    N.lib()

    w = make_workload(args.n, seed_offset=d.rank, views=args.views)
    # map build: the Gaussians stored in Morton order of their means (gs_morton_order), as the map is kept
    gm, _ = GaussianMap.from_host(w.gmap, device=d.dev).spatially_ordered()
    V, H, W = args.views, WORKLOAD["height"], WORKLOAD["width"]
    rast = Rasterizer(gm.n, V, W, H, device=d.dev)
    cams = cameras_tensor(w.cams, device=d.dev)
    tgt_rgb = torch.as_tensor(w.tgt_rgb, device=d.dev)
    tgt_depth = torch.as_tensor(w.tgt_depth, device=d.dev)
    rast.project_and_sort(gm, cams, check=True)  # sizes the pair buffer once
    out = rast.render(gm, cams, check=False)
    grads = rast.new_grads(gm)

    def step():
        grads.zero_()
        rast.render(gm, cams, check=False, out=out)
        rast.backward(gm, cams, out, tgt_rgb=tgt_rgb, tgt_depth=tgt_depth, w_rgb=w.w_rgb, w_depth=w.w_depth,
                      grads=grads)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    code, needed = rast.status()
    if code != 0:
        raise SystemExit(f"workspace status {code} after warm-up (pairs needed {needed})")
    # the step's launches and memsets replayed from one CUDA graph (the public pipeline does the same)
    from paper_2507_04004_b300.pipeline import GraphStep
    graph = GraphStep(step, d.dev)
    torch.cuda.synchronize()

    sampler = ClockSampler(d.dev.index) if d.rank == 0 else None
    time.sleep(0.6 if sampler else 0)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d.barrier()
    torch.cuda.synchronize()
    # one event per step boundary as well, for the spread of the step times
    bounds = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    t_wall0 = time.time()
    start.record()
    bounds[0].record()
    for i in range(args.steps):
        graph.replay()
        bounds[i + 1].record()
    end.record()
    end.synchronize()
    t_wall1 = time.time()
    d.barrier()
    ms_local = start.elapsed_time(end)
    ms = d.max(ms_local)
    clocks = sampler.stop(t_wall0, t_wall1) if sampler else None
    code, needed = rast.status()
    if code != 0:
        raise SystemExit(f"workspace status {code} in the timed region")

    step_times = np.array([bounds[i].elapsed_time(bounds[i + 1]) for i in range(args.steps)])
    step_pct = {q: round(float(np.percentile(step_times, int(q[1:]))), 4) for q in ("p10", "p50", "p90")}

    # per-kernel durations: the same steps again, each launch between a pair of
    # CUDA events on its stream (the library's trace hook); kept out of the
    # headline's timed region above, since the events add work of their own
    n_tr = min(args.steps, 50)
    per_step = 48
    cap = per_step * n_tr + 16
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * cap)]
    for e in evs:
        e.record()
    ids = np.zeros(cap, np.int32)
    torch.cuda.synchronize()
    N.gs_trace_start([e.cuda_event for e in evs], ids)
    for _ in range(n_tr):
        step()
    torch.cuda.synchronize()
    launches_tr = N.gs_trace_stop()
    launches = launches_tr // n_tr * args.steps  # the library's launches in the timed region
    rec = min(launches_tr, cap)
    per_kernel = {}
    for k in range(rec):
        name = N.gs_kernel_name(int(ids[k]))
        t = evs[2 * k].elapsed_time(evs[2 * k + 1])
        a = per_kernel.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += t
    total_k = sum(v[1] for v in per_kernel.values())
    kernels = {k: {"launches": v[0], "ms_total": round(v[1], 3), "ms_avg": round(v[1] / v[0], 4),
                   "per_step_ms": round(v[1] / n_tr, 4),
                   "share": round(v[1] / total_k, 4)} for k, v in sorted(per_kernel.items(), key=lambda x: -x[1][1])}
    dominant = next(iter(kernels))

    # work counters of one step (for the algorithmic roofline)
    counters = rast._view(rast.layout.counters, 8, torch.int32).cpu().numpy()
    n_visible, n_pairs, n_rows, n_listed = int(counters[2]), int(counters[1]), int(counters[4]), int(counters[5])
    k_eval = float(out.n_contrib.to(torch.float64).sum().item())
    bc = torch.zeros(args.views, 3, dtype=torch.int64, device=d.dev)
    N.gs_blend_counts(rast.cfg, rast.ws, bc, torch.cuda.current_stream(d.dev).cuda_stream)
    bc = bc.cpu().numpy().sum(0)
    k_blend = float(bc[1])
    k_skip = float(bc[0]) - k_blend
    k_tested = float(bc[2])  # list positions the forward's pixels must test (up to their stop, else all)
    p_proc = float(tile_max_prefix(out.n_contrib))
    px_step = V * H * W
    peaks = measured_peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    n_sm = torch.cuda.get_device_properties(d.dev).multi_processor_count
    issue = n_sm * 4 * sm_mhz * 1e6  # warp instructions per second (4 schedulers per SM)
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2 FLOP
    model = step_model(args.n, args.views, H * W, n_visible, n_rows, n_pairs, n_listed, p_proc, k_blend, k_skip,
                       k_tested)
    bw = peaks["hbm_gbs"] * 1e9

    def roof(k):
        bytes_, ops = model[k]
        t_s = kernels[k]["per_step_ms"] / 1e3  # all of the kernel's launches in one step
        t_mem, t_ins = bytes_ / bw, ops / 32.0 / issue
        if t_ins > t_mem:
            ach, pk, unit, bd = ops / 32.0 / t_s / 1e9, issue / 1e9, "Gwarp-instr/s", "alu"
        else:
            ach, pk, unit, bd = bytes_ / t_s / 1e9, peaks["hbm_gbs"], "GB/s", "hbm"
        return {"bound": bd, "achieved": round(ach, 3), "peak": round(pk, 2), "unit": unit,
                "frac": round(ach / pk, 4), "floor_ms": round(max(t_mem, t_ins) * 1e3, 4),
                "alg_bytes": int(bytes_), "alg_warp_instr": int(ops / 32.0), "traffic": traffic_for(k)}

    per_kernel_roof = {k: roof(k) for k in model if k in kernels}
    rf = per_kernel_roof.get(dominant)
    roofline = {"kernel": dominant, "bound": rf["bound"], "achieved": rf["achieved"], "peak": rf["peak"],
                "unit": rf["unit"], "frac": rf["frac"], "traffic": rf["traffic"],
                "peak_source": (f"instruction issue: {n_sm} SMs x 4 schedulers x {sm_mhz:.0f} MHz median SM clock "
                                "in the timed region (1 warp instruction per scheduler per clock)"
                                if rf["bound"] == "alu" else f"{peaks['source']} HBM copy bandwidth"),
                "numerator": ("algorithmic lane operations per evaluation (blended / skipped below alpha_min) "
                              "x the step's evaluations, / 32 per warp instruction"
                              if rf["bound"] == "alu" else "algorithmic bytes per launch")}
    if dominant in ("render_bwd", "render_fwd"):
        per_eval = BLEND_OPS[dominant]
        roofline["per_evaluation_ops"] = {"blended": per_eval[0], "skipped": per_eval[1]}
        # the FP32 view of the same kernel: operations x 2 for an FMA, against the FMA pipe
        fl = (k_blend * per_eval[2] + k_skip * per_eval[3]) / (kernels[dominant]["ms_avg"] / 1e3) / 1e12
        roofline["fp32_view"] = {"achieved_tflops": round(fl, 3), "peak_tflops": round(fp32_peak, 2),
                                 "frac": round(fl / fp32_peak, 4),
                                 "convention": "FLOP with FMA = 2 (blended / skipped per evaluation: "
                                               f"{per_eval[2]} / {per_eval[3]}) against 128 FP32 lanes per SM"}
    floors = sum(v["floor_ms"] for v in per_kernel_roof.values())
    step_bytes = sum(v["alg_bytes"] for v in per_kernel_roof.values())
    ms_step_local = ms_local / args.steps
    roofline_step = {
        "frac": round(floors / ms_step_local, 4),
        "floor_ms": round(floors, 4), "ms_per_step": round(ms_step_local, 4),
        "definition": "sum over the step's kernels of max(algorithmic bytes / HBM bandwidth, algorithmic "
                      "instructions / issue rate), over the measured time per step",
        "hbm_frac": round(step_bytes / (ms_step_local / 1e3) / bw, 4),
        "hbm_bytes_per_step": int(step_bytes),
        "hbm_definition": "the step's algorithmic bytes / time per step / measured HBM copy bandwidth",
    }

    # end to end: host keyframes -> device, fwd+bwd, loss back to host
    e2e = None if args.no_e2e else run_e2e(args, d, rast, gm, w, px_step)
    total_px = d.sum(px_step * args.steps)
    value = total_px / (ms / 1e3) / 1e6

    bucket = None
    if d.rank == 0 and not args.no_bucket:
        bucket = run_bucket_backward(args, rast, gm, cams, tgt_rgb, tgt_depth, w, k_blend, k_skip, issue)

    mapping_iter = None
    if d.rank == 0 and not args.no_e2e:
        mapping_iter = run_mapping_iteration(args, rast, gm, cams, w, tgt_rgb, tgt_depth)

    serving = tracking = None
    if d.rank == 0 and (args.serving_requests > 0 or args.tracking_frames > 0):
        del out, grads
        torch.cuda.empty_cache()
    if d.rank == 0 and args.tracking_frames > 0:
        tracking = run_tracking(args, d.dev)
        torch.cuda.empty_cache()
    if d.rank == 0 and args.serving_requests > 0:
        serving = run_serving(args, d.dev)

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        pix, secs, rect = oracle_sample(w, args.cpu_seconds)
        cpu = {"value": pix / secs / 1e6, "unit": "Mpix/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"view 0, centred {rect[2]}x{rect[3]} pixel rectangle, fwd+bwd in FP64 "
                         f"({secs:.1f} s)"}
        if args.cpu_seconds_one_core > 0:
            nt = O.threads()
            O.set_threads(1)
            try:
                pix1, secs1, rect1 = oracle_sample(w, args.cpu_seconds_one_core)
            finally:
                O.set_threads(nt)
            cpu["one_core"] = {"value": pix1 / secs1 / 1e6, "unit": "Mpix/s", "cores": 1,
                               "sample": f"view 0, centred {rect1[2]}x{rect1[3]} pixel rectangle ({secs1:.1f} s)"}
    if d.rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": d.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(WORKLOAD, views=args.views, n_gaussians=args.n,
                               parallelism=f"replicas x{d.world}" if d.world > 1 else "single GPU",
                               l2="inputs larger than L2: 236 MB of Gaussian parameters, 192 MB of projected records",
                               map_order="Morton order of the means (gs_morton_order at map build)",
                               launch="each timed step one replay of a CUDA graph of the step's kernels"),
                "clocks": clocks,
                "step_ms_percentiles": step_pct,
                "e2e": e2e,
                "gpu_launches": int(launches),
                "roofline": roofline,
                "roofline_step": roofline_step,
                "roofline_per_kernel": per_kernel_roof,
                "cpu_baseline": cpu,
                "mapping_iteration": mapping_iter,
                "bucket_backward": bucket,
                "tracking": tracking,
                "serving": serving,
                "kernels": kernels,
                "work": {"visible_entries": n_visible, "pairs": n_pairs, "row_items": n_rows,
                         "gaussians_listed": n_listed, "pairs_processed": p_proc,
                         "blend_evaluations": k_eval, "blend_evaluations_blended": k_blend,
                         "blend_evaluations_skipped": k_skip,
                         "forward_positions_tested": k_tested,
                         "lidar_valid_frac": [round(x, 4) for x in w.meta["depth_frac"]]}}
        print(json.dumps(line), flush=True)
    d.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
