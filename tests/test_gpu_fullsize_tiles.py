"""Tile lists and sort order at full workload sizes (needs a GPU): every
(Gaussian, tile) pair of every tile of every compared view, in order, against
the FP64 oracle's lists (every pixel of every candidate tile tested), bit-exact
outside the oracle's 1e-4 threshold margin (Sec. "Fast Tile-based Culling";
the sort on (tile, depth key, index)).  The GPU lists come from the launch
configuration bench.py times: the binning CTAs' per-window reservations and
the small / medium / long bin sorts all take part at these sizes.

Workloads: the mapping benchmark (1M Gaussians, 4 x 1920x1080); the precision
case (2M Gaussians, 8 x 1920x1080 with yaw, 1 % near-degenerate scales) with
FP32 and BF16 SH; the 500k-Gaussian 4 x 1280x720 mapping step; 6 of the 32
tracking frames (1M Gaussians, 640x512).
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import compare_tiles, host_map

pytestmark = pytest.mark.gpu

_ORACLE_LISTS = {}  # oracle lists per (workload, view): the SH storage does not change the geometry


def _gpu_lists(w, sh_bf16=False):
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    gm = GaussianMap.from_host(w.gmap, sh_bf16=sh_bf16)
    W, H = w.cams[0]["width"], w.cams[0]["height"]
    rast = Rasterizer(gm.n, len(w.cams), W, H)
    rast.project_and_sort(gm, cameras_tensor(w.cams))
    torch.cuda.synchronize()
    assert rast.status()[0] == 0
    return rast


class _CachedOracle:
    """oracle.tiles with its result kept per (workload, view)."""

    def __init__(self, oracle, key):
        self.oracle, self.key = oracle, key

    def tiles(self, m, cam):
        key = self.key
        if key not in _ORACLE_LISTS:
            _ORACLE_LISTS[key] = self.oracle.tiles(m, cam)
        return _ORACLE_LISTS[key]


def _check_views(oracle, name, w, views, sh_bf16=False):
    rast = _gpu_lists(w, sh_bf16)
    m = host_map(w.gmap, sh_bf16)
    _, count, _ = rast.tile_lists()
    c = count.cpu().numpy()
    total_margin = 0
    for v in views:
        total_margin += compare_tiles(_CachedOracle(oracle, (name, v)), m, w.cams[v], rast, v,
                                      label=f"{name} view {v}")
    return c, total_margin


def test_mapping_benchmark_workload_all_tiles(oracle):
    import bench
    w = bench.make_workload(1_000_000)
    c, nm = _check_views(oracle, "1M SH3 4x1920x1080", w, range(4))
    assert c.sum() > 10_000_000 and c.max() > 64  # warp-sorted and CTA-sorted bins both in play


@pytest.mark.parametrize("sh_bf16", [False, True])
def test_precision_2m_gaussians_8_views_all_tiles(oracle, sh_bf16):
    yaw = math.radians(20.0)
    w = synth.mapping(seed=synth.SEED_BASE + 3, n=2_000_000, width=1920, height=1080, focal=1000.0, n_views=8,
                      yaws=[0, 0, 0, 0, yaw, -yaw, yaw, -yaw], degenerate_frac=0.01)
    c, nm = _check_views(oracle, "2M SH3 8x1920x1080 (1 % degenerate)", w, range(8), sh_bf16)
    assert c.sum() > 20_000_000


def test_mapping_500k_4x720p_all_tiles(oracle):
    w = synth.mapping()
    _check_views(oracle, "500k SH3 4x1280x720", w, range(4))


def test_tracking_frames_all_tiles(oracle):
    w = synth.tracking()
    _check_views(oracle, "1M SH1 32x640x512", w, (0, 5, 11, 17, 24, 31))
