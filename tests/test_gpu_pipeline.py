"""Keyframe upload through the C ABI (needs a GPU).

gs_unpack_keyframes: colour c / 255 and the cleared, scattered depth map are
bit-exact against the host's float32 arithmetic, on ragged image sizes, with
an empty view, no depth at all, and colour only.  MappingStep: a batch
uploaded from host keyframes (8-bit image, depth pairs) gives the loss and
gradients of the same pass run on device-resident FP32 targets, also with two
batches in flight in the double buffer."""
import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import _native as N
from paper_2507_04004_b300 import synth
from paper_2507_04004_b300.pipeline import HostKeyframes, MappingStep, pack_sparse_depth

pytestmark = pytest.mark.gpu


def _unpack(rgb8, depth, with_depth=True):
    V, _, H, W = rgb8.shape
    d = lambda a: torch.as_tensor(a, device="cuda")
    rgb = torch.full((V, 3, H, W), -1.0, device="cuda")
    dep = torch.full((V, H, W), -1.0, device="cuda")
    idx, val, offs = pack_sparse_depth(depth)
    if idx.size == 0:
        idx, val = np.zeros(1, np.int32), np.zeros(1, np.float32)  # valid pointers, no entries
    st = torch.cuda.current_stream().cuda_stream
    if with_depth:
        N.gs_unpack_keyframes(d(rgb8), V, H, W, rgb, d(idx), d(val), d(offs), dep, st)
    else:
        N.gs_unpack_keyframes(d(rgb8), V, H, W, rgb, None, None, None, None, st)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), dep.cpu().numpy()


@pytest.mark.parametrize("V,H,W", [(1, 1, 1), (2, 37, 53), (3, 720, 1280)])
def test_unpack_is_exact(V, H, W):
    rng = np.random.default_rng(V * 1000 + H)
    rgb8 = rng.integers(0, 256, (V, 3, H, W), dtype=np.uint8)
    depth = np.where(rng.random((V, H, W)) < 0.04, rng.uniform(0.3, 90.0, (V, H, W)), 0.0).astype(np.float32)
    if V > 1:
        depth[0] = 0.0
    rgb, dep = _unpack(rgb8, depth)
    np.testing.assert_array_equal(rgb, rgb8.astype(np.float32) / np.float32(255.0))
    np.testing.assert_array_equal(dep, depth)


def test_unpack_misaligned_buffers():
    """Buffers off the 16-byte boundary take the byte-at-a-time path, with the
    same values."""
    rng = np.random.default_rng(8)
    V, H, W = 2, 37, 53
    rgb8 = rng.integers(0, 256, (V, 3, H, W), dtype=np.uint8)
    n = rgb8.size
    src = torch.zeros(n + 1, dtype=torch.uint8, device="cuda")
    src[1:] = torch.as_tensor(rgb8.reshape(-1), device="cuda")
    out = torch.full((n + 1,), -1.0, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    N.gs_unpack_keyframes(src[1:], V, H, W, out[1:], None, None, None, None, st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out[1:].cpu().numpy(), rgb8.reshape(-1).astype(np.float32) / np.float32(255.0))
    assert float(out[0]) == -1.0


def test_unpack_without_depth_points_and_colour_only():
    rng = np.random.default_rng(3)
    rgb8 = rng.integers(0, 256, (2, 3, 9, 11), dtype=np.uint8)
    rgb, dep = _unpack(rgb8, np.zeros((2, 9, 11), np.float32))
    assert not dep.any()
    rgb2, dep2 = _unpack(rgb8, np.zeros((2, 9, 11), np.float32), with_depth=False)
    np.testing.assert_array_equal(rgb2, rgb)
    assert np.all(dep2 == -1.0)  # untouched


def test_unpack_rejects_bad_arguments():
    x = torch.zeros(3, dtype=torch.uint8, device="cuda")
    f = torch.zeros(3, device="cuda")
    with pytest.raises(N.GsError):
        N.gs_unpack_keyframes(x, 0, 1, 1, f, None, None, None, None, 0)
    with pytest.raises(N.GsError):
        N.gs_unpack_keyframes(x, 1, 1, 1, f, torch.zeros(1, dtype=torch.int32, device="cuda"), None, None, None, 0)


def test_unpack_depth_only():
    """With no colour buffers the call writes the depth map alone (the loss then
    reads the 8-bit colour itself); one colour buffer without the other is an
    argument error."""
    rng = np.random.default_rng(4)
    V, H, W = 2, 13, 17
    depth = np.where(rng.random((V, H, W)) < 0.1, rng.uniform(0.3, 9.0, (V, H, W)), 0.0).astype(np.float32)
    idx, val, offs = pack_sparse_depth(depth)
    d = lambda a: torch.as_tensor(a, device="cuda")
    dep = torch.full((V, H, W), -1.0, device="cuda")
    N.gs_unpack_keyframes(None, V, H, W, None, d(idx), d(val), d(offs), dep, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dep.cpu().numpy(), depth)
    with pytest.raises(N.GsError):
        N.gs_unpack_keyframes(torch.zeros(3, dtype=torch.uint8, device="cuda"), 1, 1, 1, None, d(idx), d(val),
                              d(offs), dep, 0)


def test_backward_with_8bit_colour_targets():
    """gs_render_bwd_rgb8 reads the 8-bit images and takes c / 255 as the
    target: its loss and gradients are those of gs_render_bwd on the same
    targets as FP32 planes (up to the summation order of float atomics)."""
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    w = synth.mapping(n=20_000, width=160, height=96, focal=90.0, n_views=2, sh_degree=2)
    gm = GaussianMap.from_host(w.gmap)
    V, H, W = 2, 96, 160
    rast = Rasterizer(gm.n, V, W, H)
    cams = cameras_tensor(w.cams)
    out = rast.render(gm, cams)
    tgt, depth = _batch(21, w)
    tgt8 = torch.as_tensor(synth.to_uint8(tgt), device="cuda")
    assert np.array_equal(tgt8.cpu().numpy().astype(np.float32) / np.float32(255.0), tgt)
    kw = dict(tgt_depth=torch.as_tensor(depth, device="cuda"), w_rgb=w.w_rgb, w_depth=w.w_depth)
    g32 = rast.backward(gm, cams, out, tgt_rgb=torch.as_tensor(tgt, device="cuda"), **kw)
    g8 = rast.backward(gm, cams, out, tgt_rgb=tgt8, **kw)
    assert rast.status()[0] == 0
    np.testing.assert_allclose(g8.loss.cpu().numpy(), g32.loss.cpu().numpy(), rtol=1e-6)
    for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest", "pose"):
        a, b = getattr(g8, k).cpu().numpy(), getattr(g32, k).cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=k)
    bucket = Rasterizer(gm.n, V, W, H, backward="bucket")
    out_b = bucket.render(gm, cams)
    with pytest.raises(ValueError):
        bucket.backward(gm, cams, out_b, tgt_rgb=tgt8, **kw)


def _batch(seed, w):
    rng = np.random.default_rng(seed)
    V, _, H, W = w.tgt_rgb.shape
    tgt = synth.quantize_8bit(rng.random((V, 3, H, W)))
    depth = np.where(rng.random((V, H, W)) < 0.05, rng.uniform(1.0, 12.0, (V, H, W)), 0.0).astype(np.float32)
    return tgt, depth


@pytest.mark.parametrize("graphs,backward", [(True, "pixel"), (False, "pixel"), (True, "bucket")])
def test_mapping_step_matches_device_resident_pass(graphs, backward):
    """The host-fed step (eager, or replayed from a CUDA graph per upload
    slot; the pixel backward reading the 8-bit colour, the bucket backward the
    unpacked planes) gives the loss and gradients of the device-resident pass."""
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    w = synth.mapping(n=20_000, width=160, height=96, focal=90.0, n_views=2, sh_degree=2)
    gm = GaussianMap.from_host(w.gmap)
    V, H, W = 2, 96, 160
    rast = Rasterizer(gm.n, V, W, H, backward=backward)
    cams = cameras_tensor(w.cams)
    rast.project_and_sort(gm, cams, check=True)
    batches = [_batch(s, w) for s in (11, 12)]

    def resident(tgt, depth):
        out = rast.render(gm, cams, check=False)
        g = rast.backward(gm, cams, out, tgt_rgb=torch.as_tensor(tgt, device="cuda"),
                          tgt_depth=torch.as_tensor(depth, device="cuda"), w_rgb=w.w_rgb, w_depth=w.w_depth)
        return {k: getattr(g, k).cpu().numpy() for k in ("loss", "mean", "sh_dc", "logit_opacity", "pose")}

    refs = [resident(*b) for b in batches]
    ms = MappingStep(rast, gm, w.w_rgb, w.w_depth, graphs=graphs)
    kfs = [HostKeyframes.from_dense(synth.to_uint8(t), d, cams.cpu()) for t, d in batches]
    slots = [ms.upload(kf) for kf in kfs]          # both batches in flight
    assert ms.h2d_bytes == kfs[1].nbytes()
    for slot, ref in list(zip(slots, refs)) * 2:  # second round: graphs already captured
        loss = ms.step(slot)
        torch.cuda.synchronize()
        np.testing.assert_allclose(loss.numpy(), ref["loss"], rtol=1e-5)
        for k in ("mean", "sh_dc", "logit_opacity", "pose"):
            got = getattr(ms.grads, k).cpu().numpy()
            np.testing.assert_allclose(got, ref[k], rtol=1e-4, atol=1e-6 * np.abs(ref[k]).max(), err_msg=k)
