"""The allocation-free forward render (gs_render_fwd_noalloc) gives the same
images as the workspace path.

Callers that cannot call cudaMalloc (a host framework that owns all device
memory, a real-time loop that cannot take cudaMalloc's device synchronisation)
use this entry point; its scratch is a fixed device array inside the library.
This file is named to be collected last.  Both calls below go through the C
ABI and reuse the same scratch array, so the second one also shows that what
the first call left behind does not leak into its result.
"""
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import IMG_TOL


def _scenes():
    # a larger scene first, then a smaller one at another resolution
    a = synth.mapping(n=40000, width=200, height=120, focal=110.0, n_views=2)
    b = synth.tiny(n=1500, width=96, height=72)
    return [(a.gmap, a.cams), (b.gmap, b.cams)]


@pytest.mark.gpu
def test_noalloc_matches_workspace_path_on_two_calls():
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor, make_config
    cfg = make_config()
    for g, cams in _scenes():
        gm = GaussianMap.from_host(g)
        V, W, H = len(cams), cams[0]["width"], cams[0]["height"]
        ct = cameras_tensor(cams)
        ref = Rasterizer(gm.n, V, W, H).render(gm, ct)
        f = dict(device="cuda", dtype=torch.float32)
        rgb, depth, opac, tf = (torch.full((V, 3, H, W), -1.0, **f), torch.full((V, H, W), -1.0, **f),
                                torch.full((V, H, W), -1.0, **f), torch.full((V, H, W), -1.0, **f))
        nc = torch.full((V, H, W), -1, device="cuda", dtype=torch.int32)
        status = torch.full((1,), -1, device="cuda", dtype=torch.int32)
        code = N.gs_render_fwd_noalloc(gm.struct(), ct, N.gs_frame(V, W, H), cfg, rgb, depth, opac, tf, nc, status,
                                       torch.cuda.current_stream().cuda_stream)
        assert code == N.GS_OK
        torch.cuda.synchronize()
        assert int(status.item()) == N.GS_OK
        for a, b in ((rgb, ref.rgb), (depth, ref.depth), (opac, ref.opac), (tf, ref.t_final)):
            err = float((a - b).abs().max())
            assert err <= IMG_TOL, err
        assert torch.equal(nc, ref.n_contrib)


def _noalloc(N, gm, ct, V, W, H, cfg, with_planes=True):
    f = dict(device="cuda", dtype=torch.float32)
    planes = ((torch.full((V, 3, H, W), -1.0, **f), torch.full((V, H, W), -1.0, **f),
               torch.full((V, H, W), -1.0, **f)) if with_planes else (None, None, None))
    tf = torch.full((V, H, W), -1.0, **f)
    nc = torch.full((V, H, W), -1, device="cuda", dtype=torch.int32)
    status = torch.full((1,), -1, device="cuda", dtype=torch.int32)
    code = N.gs_render_fwd_noalloc(gm.struct(), ct, N.gs_frame(V, W, H), cfg, *planes, tf, nc, status,
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return code, int(status.item()), planes, tf, nc


@pytest.mark.gpu
def test_noalloc_without_colour_depth_and_opacity_planes():
    """rgb, depth and opac may be NULL: t_final and n_contrib still match the
    workspace path."""
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor, make_config
    w = synth.tiny(n=1500, width=96, height=72)
    gm = GaussianMap.from_host(w.gmap)
    ct = cameras_tensor(w.cams)
    ref = Rasterizer(gm.n, 1, 96, 72).render(gm, ct)
    code, status, _, tf, nc = _noalloc(N, gm, ct, 1, 96, 72, make_config(), with_planes=False)
    assert code == N.GS_OK and status == N.GS_OK
    assert float((tf - ref.t_final).abs().max()) <= IMG_TOL
    assert torch.equal(nc, ref.n_contrib)


@pytest.mark.gpu
def test_noalloc_pair_overflow_reports_capacity_and_background():
    """A batch whose (Gaussian, tile) pairs exceed what the array leaves after
    the per-Gaussian parts: the device status is GS_ERR_CAPACITY and the images
    are background only; a following call that fits is correct again."""
    import numpy as np
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor, make_config
    rng = np.random.default_rng(synth.SEED_BASE + 77)
    # 200k large Gaussians at 256x256: the per-Gaussian workspace leaves room
    # for about 3M pairs; the scene has several million more
    g = synth.random_map(rng, 200_000, (-4, -4, 2), (4, 4, 12), 0, log_scale_mean=-0.5, log_scale_std=0.2)
    W = H = 256
    cam = synth.camera(np.eye(3), np.zeros(3), 100.0, 100.0, W / 2, H / 2, W, H)
    gm = GaussianMap.from_host(g)
    ct = cameras_tensor([cam])
    cfg = make_config()
    # the pair capacity the call derives: the largest whose workspace layout fits the array
    frame = N.gs_frame(1, W, H)
    lo, hi = 1, N.GS_NOALLOC_SCRATCH_BYTES
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if N.gs_workspace_size(g.n, frame, mid) <= N.GS_NOALLOC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    cap = lo
    code, status, (rgb, depth, opac), tf, nc = _noalloc(N, gm, ct, 1, W, H, cfg)
    assert code == N.GS_OK
    assert status == N.GS_ERR_CAPACITY, status
    assert bool((tf == 1.0).all()) and bool((nc == 0).all())
    assert float(rgb.abs().max()) == 0.0 and float(depth.abs().max()) == 0.0 and float(opac.abs().max()) == 0.0
    # the workspace path needs more pairs than the array could hold
    rast = Rasterizer(gm.n, 1, W, H)
    rast.render(gm, ct)
    code, needed = rast.status()
    assert code == N.GS_OK and needed > cap, (needed, cap)
    # the next call that fits starts from a clean status
    w = synth.tiny(n=1500, width=96, height=72)
    gs = GaussianMap.from_host(w.gmap)
    cs = cameras_tensor(w.cams)
    ref = Rasterizer(gs.n, 1, 96, 72).render(gs, cs)
    code, status, (rgb, _, _), tf, nc = _noalloc(N, gs, cs, 1, 96, 72, cfg)
    assert code == N.GS_OK and status == N.GS_OK
    assert float((rgb - ref.rgb).abs().max()) <= IMG_TOL
    assert torch.equal(nc, ref.n_contrib)


def test_noalloc_rejects_requests_larger_than_its_array():
    from paper_2507_04004_b300 import build as B
    B.build()
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import make_config

    class Addr:  # a non-null device address that is never dereferenced: the call rejects first
        def data_ptr(self):
            return 0x1000

    n = 1_000_000  # 4 views x 1M Gaussians x 108 B of per-Gaussian workspace >> 64 MiB
    m = N.gs_map(n, 0, 0, 0x1000, 0x1000, 0x1000, 0x1000, 0x1000, None)
    code = N.gs_render_fwd_noalloc(m, Addr(), N.gs_frame(4, 1920, 1080), make_config(), None, None, None, Addr(),
                                   Addr(), Addr(), 0)
    assert code == N.GS_ERR_UNSUPPORTED
