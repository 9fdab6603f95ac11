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
