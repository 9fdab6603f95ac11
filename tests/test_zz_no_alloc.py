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
