"""Spatial storage order of the map (needs a GPU): gs_morton_order against
the Morton codes recomputed on the host in the same FP32 operations (the
permutation must be their stable sort), gs_permute_rows against indexing,
and the rasterizer's invariance to the storage order (images bit-identical,
gradients the permuted ones)."""
import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import GRAD_TOL, rel_err

pytestmark = pytest.mark.gpu


def _spread3(q):
    out = np.zeros_like(q, dtype=np.uint64)
    for b in range(10):
        out |= ((q.astype(np.uint64) >> b) & 1) << (3 * b)
    return out


def _host_codes(mean):
    """Codes from the definition in gs.h: q = floor((m - lo) * (1024 / (hi - lo))) in FP32."""
    m = np.asarray(mean, np.float32)
    q = np.zeros(m.shape, np.uint64)
    for a in range(3):
        fin = np.isfinite(m[a])
        lo, hi = m[a][fin].min(), m[a][fin].max()
        ext = np.float32(hi - lo)
        scale = np.float32(np.float32(1024.0) / ext) if ext > 0 else np.float32(0.0)
        t = np.floor(np.float32(m[a] - lo) * scale).astype(np.float32)
        t = np.where(fin, t, 0.0)
        q[a] = np.clip(t, 0, 1023).astype(np.uint64)
    return (_spread3(q[0]) << 2) | (_spread3(q[1]) << 1) | _spread3(q[2])


@pytest.mark.parametrize("n", [1, 777, 5000, 300_001])
def test_morton_order_is_the_stable_sort_of_the_codes(n):
    from paper_2507_04004_b300.raster import GaussianMap, morton_order
    rng = np.random.default_rng(n)
    g = synth.random_map(rng, n, (-30, -10, -30), (30, 10, 30), 0)
    if n > 10:
        g.mean[:, 3] = g.mean[:, 7]      # equal codes: index order
        g.mean[0, 11] = np.nan           # a non-finite mean gets code 0 on that axis
        g.mean[:, 5] = g.mean.max(axis=1)  # the box corner: q = 1023
    gm = GaussianMap.from_host(g)
    perm = morton_order(gm).cpu().numpy().astype(np.int64)
    codes = _host_codes(g.mean)
    want = np.lexsort((np.arange(n), codes))
    np.testing.assert_array_equal(perm, want)


def test_permute_rows_float_and_bf16():
    from paper_2507_04004_b300.raster import permute_rows
    rng = np.random.default_rng(3)
    n = 10_007
    perm = torch.as_tensor(rng.permutation(n).astype(np.int32), device="cuda")
    a = torch.as_tensor(rng.normal(size=(15, 3, n)).astype(np.float32), device="cuda")
    assert torch.equal(permute_rows(a, perm), a[..., perm.long()])
    b = a.to(torch.bfloat16)
    assert torch.equal(permute_rows(b, perm), b[..., perm.long()])


def test_rendering_is_invariant_to_the_storage_order():
    """The same map in Morton order: images and contributor counts identical,
    the loss equal, gradients the permuted gradients of the original order."""
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor, permute_rows
    w = synth.mapping(n=40_000, width=200, height=120, focal=110.0, n_views=2)
    gm = GaussianMap.from_host(w.gmap)
    gs, perm = gm.spatially_ordered()
    ct = cameras_tensor(w.cams)
    t = lambda x: torch.as_tensor(x, device="cuda")
    res = []
    for m in (gm, gs):
        r = Rasterizer(m.n, 2, 200, 120)
        out = r.render(m, ct)
        g = r.backward(m, ct, out, tgt_rgb=t(w.tgt_rgb[:, :, :120, :200]), tgt_depth=t(w.tgt_depth[:, :120, :200]),
                       w_rgb=w.w_rgb, w_depth=w.w_depth)
        torch.cuda.synchronize()
        res.append((out, g))
    (o0, g0), (o1, g1) = res
    for a, b in ((o0.rgb, o1.rgb), (o0.depth, o1.depth), (o0.t_final, o1.t_final), (o0.n_contrib, o1.n_contrib)):
        assert torch.equal(a, b)
    np.testing.assert_allclose(g0.loss.cpu().numpy(), g1.loss.cpu().numpy(), rtol=1e-6)
    for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest"):
        want = permute_rows(getattr(g0, k), perm).cpu().numpy()
        assert rel_err(getattr(g1, k).cpu().numpy(), want) <= 1e-5, k
    assert rel_err(g1.pose.cpu().numpy(), g0.pose.cpu().numpy()) <= 1e-5
