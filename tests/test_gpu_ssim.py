"""D-SSIM through the C ABI (needs a GPU) against the FP64 oracle: loss and
gradient on ragged multi-tile images, accumulation into existing buffers,
and a 1920x1080 view checked on pixel rectangles (SSIM at a pixel depends on
the images within 5 pixels, its gradient within 10, so the oracle evaluated
on a crop is exact away from the crop's border)."""
import numpy as np
import pytest
import torch

from oracle import ssim as S
from paper_2507_04004_b300 import synth
from tests.gpu_cases import GRAD_TOL, rel_err

pytestmark = pytest.mark.gpu


def _images(rng, V, H, W):
    x = np.stack([synth.smooth_target(rng, H, W) for _ in range(V)]).astype(np.float32)
    y = np.clip(x + 0.15 * rng.normal(size=x.shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("V,H,W", [(2, 37, 53), (1, 96, 128), (3, 70, 33)])
def test_dssim_loss_and_gradient(V, H, W):
    from paper_2507_04004_b300.raster import DSSIM
    rng = np.random.default_rng(H * W)
    x, y = _images(rng, V, H, W)
    t = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    loss = t(np.full(V, 0.25, np.float32))
    base = rng.normal(size=x.shape).astype(np.float32)
    grad = t(base)
    DSSIM(V, H, W)(t(x), t(y), 0.7, loss=loss, dl_dimg=grad)
    loss, grad = loss.cpu().numpy(), grad.cpu().numpy() - base
    for v in range(V):
        assert loss[v] == pytest.approx(0.25 + 0.7 * S.dssim(x[v], y[v]), abs=2e-6)
        go = 0.7 * S.dssim_grad(x[v], y[v])
        assert rel_err(grad[v], go) <= GRAD_TOL


def test_dssim_of_identical_images_is_zero():
    from paper_2507_04004_b300.raster import DSSIM
    rng = np.random.default_rng(3)
    x, _ = _images(rng, 2, 64, 80)
    t = torch.as_tensor(x, device="cuda")
    loss = torch.zeros(2, device="cuda")
    grad = torch.zeros_like(t)
    DSSIM(2, 64, 80)(t, t.clone(), 1.0, loss=loss, dl_dimg=grad)
    assert np.abs(loss.cpu().numpy()).max() < 1e-5
    # exact zero in real arithmetic; FP32 cancellation leaves ~1e-4 of the gradient scale 1 / (3 H W)
    assert np.abs(grad.cpu().numpy()).max() < 1e-3 / (3 * 64 * 80)


def test_dssim_1080p_on_rectangles():
    from paper_2507_04004_b300.raster import DSSIM
    rng = np.random.default_rng(4)
    H, W = 1080, 1920
    x, y = _images(rng, 1, H, W)
    tx, ty = torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda")
    grad = torch.zeros_like(tx)
    loss = torch.zeros(1, device="cuda")
    DSSIM(1, H, W)(tx, ty, 1.0, loss=loss, dl_dimg=grad)
    g = grad.cpu().numpy()[0]
    n_full = 3 * H * W
    for (x0, y0, rw, rh) in [(0, 0, 40, 32), (936, 520, 48, 40), (1890, 1052, 30, 28)]:
        # crop with a 10-pixel margin where the image continues (zero padding at the image border either way)
        cx0, cy0 = max(0, x0 - 10), max(0, y0 - 10)
        cx1, cy1 = min(W, x0 + rw + 10), min(H, y0 + rh + 10)
        xc, yc = x[0][:, cy0:cy1, cx0:cx1], y[0][:, cy0:cy1, cx0:cx1]
        go = S.dssim_grad(xc, yc) * (xc.size / n_full)
        sl = (slice(None), slice(y0 - cy0, y0 - cy0 + rh), slice(x0 - cx0, x0 - cx0 + rw))
        assert rel_err(g[:, y0:y0 + rh, x0:x0 + rw], go[sl]) <= GRAD_TOL
        sm = S.ssim_map(xc, yc)
        inner = sm[:, (y0 - cy0):(y0 - cy0 + rh), (x0 - cx0):(x0 - cx0 + rw)]
        assert np.isfinite(inner).all()
    # the loss against the oracle on the whole view (FP64 SSIM map, a few seconds)
    assert loss.item() == pytest.approx(S.dssim(x[0], y[0]), abs=5e-6)


@pytest.mark.parametrize("V,H,W", [(2, 50, 100), (1, 1080, 1920)])
def test_dssim_tma_and_cpasync_staging_agree(V, H, W):
    """Rows of 16-byte stride on 16-byte aligned buffers are staged by TMA,
    other buffers element by element; the arithmetic after staging is the
    same, so the two agree bit for bit.  The second staging is forced by
    offsetting every buffer by one float."""
    from paper_2507_04004_b300.raster import DSSIM
    rng = np.random.default_rng(W + 7)
    x, y = _images(rng, V, H, W)
    base = rng.normal(size=x.shape).astype(np.float32)
    n = x.size

    def run(offset):
        buf = torch.zeros(3 * (n + 4), device="cuda")
        parts = [buf[k * (n + 4) + offset:k * (n + 4) + offset + n].view(x.shape) for k in range(3)]
        parts[0].copy_(torch.as_tensor(x))
        parts[1].copy_(torch.as_tensor(y))
        parts[2].copy_(torch.as_tensor(base))
        loss = torch.zeros(V, device="cuda")
        DSSIM(V, H, W)(parts[0], parts[1], 0.5, loss=loss, dl_dimg=parts[2])
        return loss.cpu().numpy(), parts[2].cpu().numpy()

    l0, g0 = run(0)
    l1, g1 = run(1)
    assert np.array_equal(g0, g1)
    # the loss sums per-CTA partials with atomics: equal up to summation order
    np.testing.assert_allclose(l0, l1, rtol=0, atol=1e-6)
    if H * W <= 10000:
        for v in range(V):
            assert l0[v] == pytest.approx(0.5 * S.dssim(x[v], y[v]), abs=2e-6)
            assert rel_err(g0[v] - base[v], 0.5 * S.dssim_grad(x[v], y[v])) <= GRAD_TOL
