"""Map expansion through the C ABI (needs a GPU): the points selected for a
keyframe against the FP64 selection on the same opacity map (rendered by the
oracle), the initial values of the new Gaussians, and, end to end, that the
grown map covers pixels the old one left empty."""
import math

import numpy as np
import pytest
import torch

from oracle import expand as E
from paper_2507_04004_b300 import synth
from tests.gpu_cases import host_map

pytestmark = pytest.mark.gpu


def _points(rng, P):
    # camera-frame points spread over and beyond the tiny scene's frustum, some behind the camera
    xyz = np.stack([rng.uniform(-8, 8, P), rng.uniform(-6, 6, P), rng.uniform(-3, 14, P)])
    return xyz, rng.random((3, P))


def test_selection_and_initial_values(oracle):
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import GaussianMap, cameras_tensor, expand_map
    w = synth.tiny()
    m = host_map(w.gmap)
    cam = w.cams[0]
    opac = oracle.render(m, cam)["opac"].astype(np.float32)
    assert (opac < 0.99).mean() > 0.05 and (opac >= 0.99).mean() > 0.05
    rng = np.random.default_rng(40)
    P = 20000
    pts, rgb = _points(rng, P)
    pts32, rgb32 = pts.astype(np.float32), rgb.astype(np.float32)
    want, border = E.select_points(pts32.astype(np.float64), cam, opac.astype(np.float64), tau=0.99)
    gm = GaussianMap.from_host(w.gmap)
    t = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    grown, idx = expand_map(gm, t(pts32), t(rgb32), cameras_tensor([cam]), t(opac), tau=0.99, init_opacity=0.1)
    got = idx.cpu().numpy()
    # FP32 and FP64 may place a projection within 1e-4 px of a pixel border on different sides
    ambiguous = set(np.nonzero(border < 1e-4)[0].tolist())
    diff = set(got.tolist()) ^ set(want.tolist())
    assert diff <= ambiguous, sorted(diff - ambiguous)[:10]
    assert len(got) > 1000 and np.all(np.diff(got) > 0)  # ascending: the input order is kept
    n0 = gm.n
    assert grown.n == n0 + len(got)
    for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest"):
        np.testing.assert_array_equal(getattr(grown, k)[..., :n0].cpu().numpy(), getattr(gm, k).cpu().numpy())
    new = lambda k: getattr(grown, k)[..., n0:].cpu().numpy()
    np.testing.assert_array_equal(new("mean"), pts32[:, got])
    z = pts32[2, got].astype(np.float64)  # identity pose: depth = z
    np.testing.assert_allclose(new("log_scale"), np.log(2 * z / cam["fx"])[None].repeat(3, 0), rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(new("quat"), np.array([[1.0], [0.0], [0.0], [0.0]]) * np.ones((1, len(got))))
    np.testing.assert_allclose(new("logit_opacity"), math.log(0.1 / 0.9), rtol=1e-6)
    np.testing.assert_allclose(0.5 + 0.28209479177387814 * new("sh_dc"), rgb32[:, got], atol=1e-6)


def test_expansion_fills_empty_pixels():
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor, expand_map
    w = synth.tiny()
    gm = GaussianMap.from_host(w.gmap)
    cams = cameras_tensor(w.cams)
    r = Rasterizer(gm.n, 1, 128, 96)
    o0 = r.render(gm, cams).opac[0].clone()
    rng = np.random.default_rng(41)
    # LiDAR-like points on a wall behind the scene, one per pixel ray
    ys, xs = np.mgrid[0:96, 0:128]
    z = 14.0
    pts = np.stack([(xs + 0.5 - 64) / 100 * z, (ys + 0.5 - 48) / 100 * z, np.full(xs.shape, z)]).reshape(3, -1)
    t = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda").contiguous()
    grown, idx = expand_map(gm, t(pts), t(rng.random(pts.shape)), cams, o0.contiguous(), tau=0.99, init_opacity=0.9)
    empty = (o0 < 0.99).cpu().numpy().reshape(-1)
    assert np.array_equal(np.sort(idx.cpu().numpy()), np.nonzero(empty)[0])  # one point per masked pixel
    r2 = Rasterizer(grown.n, 1, 128, 96)
    o1 = r2.render(grown, cams).opac[0].cpu().numpy().reshape(-1)
    assert np.all(o1 >= o0.cpu().numpy().reshape(-1) - 1e-6)
    assert np.mean(o1[empty] > 0.5) > 0.95
