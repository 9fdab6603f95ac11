"""Batches of more than 32 views (needs a GPU).

The projection holds the cameras of up to 32 views at a time in shared
memory and restages them, between barriers, for every further chunk of views.
Views are independent all the way through, so rendering 40 views in one batch
(two chunks) must give each view what rendering them in batches of 20 (one
chunk each) gives."""
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import IMG_TOL

pytestmark = pytest.mark.gpu


def test_forty_views_in_one_batch_match_two_batches_of_twenty():
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    w = synth.mapping(n=20000, width=96, height=64, focal=55.0, n_views=40, sh_degree=2)
    gm = GaussianMap.from_host(w.gmap)
    H, W = 64, 96
    full = Rasterizer(gm.n, 40, W, H).render(gm, cameras_tensor(w.cams))
    for v0 in (0, 20):
        part = Rasterizer(gm.n, 20, W, H).render(gm, cameras_tensor(w.cams[v0:v0 + 20]))
        sl = slice(v0, v0 + 20)
        assert torch.equal(full.n_contrib[sl], part.n_contrib)
        for a, b in ((full.rgb[sl], part.rgb), (full.depth[sl], part.depth), (full.opac[sl], part.opac),
                     (full.t_final[sl], part.t_final)):
            assert float((a - b).abs().max()) <= IMG_TOL
    # the scene is seen: some pixels of every view are covered
    assert bool((full.opac.flatten(1).amax(1) > 0.1).all())


@pytest.mark.parametrize("n", [3000, 24])
def test_pose_only_backward_over_many_small_views(n):
    """The pose-only backward runs one thread per sorted visible entry, each CTA
    over a contiguous share of them.  With 300 small views the batch has more
    views than the full backward keeps in shared memory, and with a map of 24
    Gaussians a share of 256 entries spans many views, past the ones it sums
    in shared memory.  The pose gradient of the pose-only backward equals that
    of the full one, view by view."""
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    V, H, W = 300, 24, 32
    w = synth.mapping(n=n, width=W, height=H, focal=20.0, n_views=V, sh_degree=1)
    gm = GaussianMap.from_host(w.gmap)
    cams = cameras_tensor(w.cams)
    rast = Rasterizer(gm.n, V, W, H)
    out = rast.render(gm, cams)
    tgt = torch.as_tensor(w.tgt_rgb, device="cuda")
    full = rast.backward(gm, cams, out, tgt_rgb=tgt, w_rgb=1.0)
    pose_only = rast.backward(gm, cams, out, tgt_rgb=tgt, w_rgb=1.0, params=False)
    assert rast.status()[0] == 0
    a, b = pose_only.pose.double(), full.pose.double()
    assert int((b.abs().amax(1) > 0).sum()) > V // 10  # views that see something
    scale = b.abs().amax(1, keepdim=True).clamp_min(1e-30)
    assert float(((a - b).abs() / scale).max()) <= 1e-4
