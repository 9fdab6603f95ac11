"""Parity at full workload sizes, in the launch configuration bench.py times
(needs a GPU).  The oracle computes sampled pixel rectangles one by one;
gradients are compared through pixel adjoints that are non-zero only inside
those rectangles, which the oracle back-propagates exactly.

Workloads: the mapping benchmark (1M Gaussians, SH 3, 4 x 1920x1080); the
precision case (2M Gaussians, SH 3 in BF16 and FP32, 8 views of 1920x1080,
1 % of Gaussians with one log-scale at -8); the tracking case (1M Gaussians,
SH 1, 32 frames of 640x512, Jacobian rows of the 20k highest-gradient pixels).
"""
import math

import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import GRAD_TOL, IMG_TOL, assert_grads_close, grads_to_numpy, host_map, rel_err

pytestmark = pytest.mark.gpu

GRAD_KEYS = ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest")
RECTS_1080 = [(0, 0, 40, 32), (936, 520, 48, 40), (1890, 1052, 30, 28)]  # corner, centre, ragged edge


def _render(w, sh_bf16=False):
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    gm = GaussianMap.from_host(w.gmap, sh_bf16=sh_bf16)
    W, H = w.cams[0]["width"], w.cams[0]["height"]
    rast = Rasterizer(gm.n, len(w.cams), W, H)
    ct = cameras_tensor(w.cams)
    out = rast.render(gm, ct)
    torch.cuda.synchronize()
    return rast, gm, ct, out


def _image_errors(oracle, m, cam, out, v, rect):
    x0, y0, rw, rh = rect
    o = oracle.render(m, cam, rect=rect)
    ok = o["flags"] == 0
    rgb = out.rgb[v, :, y0:y0 + rh, x0:x0 + rw].cpu().numpy()
    dep = out.depth[v, y0:y0 + rh, x0:x0 + rw].cpu().numpy()
    opa = out.opac[v, y0:y0 + rh, x0:x0 + rw].cpu().numpy()
    e_rgb = np.abs(rgb - o["rgb"])[:, ok]
    e_o = np.abs(opa - o["opac"])[ok]
    e_d = np.abs(dep - o["depth"])[ok]
    return e_rgb, e_o, e_d, float(max(1.0, np.abs(o["depth"]).max())), float(ok.mean())


def _rect_adjoints(shape_v, H, W, views, rects, seed):
    rng = np.random.default_rng(seed)
    V = shape_v
    er = np.zeros((V, 3, H, W), np.float32)
    ed = np.zeros((V, H, W), np.float32)
    eo = np.zeros((V, H, W), np.float32)
    for v in views:
        for (x0, y0, rw, rh) in rects:
            er[v, :, y0:y0 + rh, x0:x0 + rw] = rng.normal(size=(3, rh, rw))
            ed[v, y0:y0 + rh, x0:x0 + rw] = 0.02 * rng.normal(size=(rh, rw))
            eo[v, y0:y0 + rh, x0:x0 + rw] = rng.normal(size=(rh, rw))
    return er, ed, eo


def _oracle_rect_grads(oracle, m, cams, views, rects, er, ed, eo):
    tot = None
    pose = np.zeros((len(cams), 6))
    for v in views:
        for rect in rects:
            o = oracle.backward(m, [cams[v]], ext_rgb=er[v:v + 1], ext_depth=ed[v:v + 1], ext_opac=eo[v:v + 1],
                                rect=rect)
            pose[v] += o["pose"][0]
            if tot is None:
                tot = {k: o[k].copy() for k in GRAD_KEYS}
            else:
                for k in GRAD_KEYS:
                    tot[k] += o[k]
    tot["pose"] = pose
    return tot


def test_mapping_benchmark_workload_sampled(oracle):
    import bench
    w = bench.make_workload(1_000_000)
    m = host_map(w.gmap)
    rast, gm, ct, out = _render(w)
    assert rast.status()[0] == 0
    for v in (0, 3):
        for rect in RECTS_1080:
            e_rgb, e_o, e_d, dscale, okf = _image_errors(oracle, m, w.cams[v], out, v, rect)
            assert okf > 0.9
            assert e_rgb.max() <= IMG_TOL and e_o.max() <= IMG_TOL and e_d.max() <= IMG_TOL * dscale, (v, rect)
    H, W = 1080, 1920
    er, ed, eo = _rect_adjoints(4, H, W, (0, 3), RECTS_1080, 17)
    t = lambda a: torch.as_tensor(a, device="cuda")
    g = grads_to_numpy(rast.backward(gm, ct, out, dl_drgb=t(er), dl_ddepth=t(ed), dl_dopac=t(eo)))
    o = _oracle_rect_grads(oracle, m, w.cams, (0, 3), RECTS_1080, er, ed, eo)
    assert_grads_close(g, o, GRAD_KEYS, label="1M SH3 4x1080p, sampled rectangles")
    for v in (0, 3):
        assert rel_err(g["pose"][v], o["pose"][v]) <= GRAD_TOL, v
    assert np.abs(g["pose"][1]).max() == 0 and np.abs(g["pose"][2]).max() == 0


RECTS_720 = [(0, 0, 40, 32), (616, 340, 48, 40), (1250, 692, 30, 28)]  # corner, centre, ragged edge


def test_mapping_500k_4x720p_sampled(oracle):
    """The 500k-Gaussian mapping step (SH 3, 4 keyframes of 1280x720, fx = 700,
    LiDAR depth, 0.8 L1 colour + 0.2 L1 depth): images and gradients against
    the oracle on sampled rectangles, and the fused loss backward against the
    external-adjoint backward fed with the loss's own pixel adjoints."""
    w = synth.mapping()
    m = host_map(w.gmap)
    rast, gm, ct, out = _render(w)
    assert rast.status()[0] == 0
    for v in (0, 3):
        for rect in RECTS_720:
            e_rgb, e_o, e_d, dscale, okf = _image_errors(oracle, m, w.cams[v], out, v, rect)
            assert okf > 0.9
            assert e_rgb.max() <= IMG_TOL and e_o.max() <= IMG_TOL and e_d.max() <= IMG_TOL * dscale, (v, rect)
    H, W = 720, 1280
    er, ed, eo = _rect_adjoints(4, H, W, (0, 3), RECTS_720, 29)
    t = lambda a: torch.as_tensor(a, device="cuda")
    g = grads_to_numpy(rast.backward(gm, ct, out, dl_drgb=t(er), dl_ddepth=t(ed), dl_dopac=t(eo)))
    o = _oracle_rect_grads(oracle, m, w.cams, (0, 3), RECTS_720, er, ed, eo)
    assert_grads_close(g, o, GRAD_KEYS, label="500k SH3 4x720p, sampled rectangles")
    for v in (0, 3):
        assert rel_err(g["pose"][v], o["pose"][v]) <= GRAD_TOL, v

    # fused loss == external adjoints of the same loss (a property at any size)
    tr, td = t(w.tgt_rgb), t(w.tgt_depth)
    gf = rast.backward(gm, ct, out, tgt_rgb=tr, tgt_depth=td, w_rgb=w.w_rgb, w_depth=w.w_depth)
    r = out.rgb - tr
    dC = w.w_rgb * torch.sign(r) / (3.0 * H * W)
    nd = (td > 0).flatten(1).sum(1).to(torch.float32).view(4, 1, 1)
    valid = (td > 0) & (out.opac > 0)
    O = torch.where(valid, out.opac, torch.ones_like(out.opac))
    sg = torch.where(valid, torch.sign(out.depth / O - td), torch.zeros_like(td))
    dD = w.w_depth * sg / (O * nd)
    dO = -w.w_depth * sg * out.depth / (O * O * nd)
    ge = rast.backward(gm, ct, out, dl_drgb=dC.contiguous(), dl_ddepth=dD.contiguous(), dl_dopac=dO.contiguous())
    gf, ge = grads_to_numpy(gf), grads_to_numpy(ge)
    for k in GRAD_KEYS + ("pose",):
        assert rel_err(gf[k], ge[k]) <= GRAD_TOL, k
    loss = (w.w_rgb * r.abs().flatten(1).mean(1)
            + w.w_depth * (torch.where(valid, (out.depth / O - td).abs(), torch.zeros_like(td)).flatten(1).sum(1)
                           / nd.view(4)))
    np.testing.assert_allclose(gf["loss"], loss.cpu().numpy(), rtol=1e-4)


@pytest.mark.parametrize("sh_bf16", [True, False])
def test_precision_2m_gaussians_8_views_sampled(oracle, sh_bf16, capsys):
    yaw = math.radians(20.0)
    w = synth.mapping(seed=synth.SEED_BASE + 3, n=2_000_000, width=1920, height=1080, focal=1000.0, n_views=8,
                      yaws=[0, 0, 0, 0, yaw, -yaw, yaw, -yaw], degenerate_frac=0.01)
    m = host_map(w.gmap, sh_bf16)
    rast, gm, ct, out = _render(w, sh_bf16)
    assert rast.status()[0] == 0
    worst = dict(rgb=0.0, opac=0.0, depth=0.0)
    means = dict(rgb=[], opac=[], depth=[])
    for v in (0, 5):
        for rect in RECTS_1080:
            e_rgb, e_o, e_d, dscale, okf = _image_errors(oracle, m, w.cams[v], out, v, rect)
            assert okf > 0.9
            worst["rgb"] = max(worst["rgb"], float(e_rgb.max()))
            worst["opac"] = max(worst["opac"], float(e_o.max()))
            worst["depth"] = max(worst["depth"], float(e_d.max() / dscale))
            means["rgb"].append(float(e_rgb.mean())); means["opac"].append(float(e_o.mean()))
            means["depth"].append(float(e_d.mean() / dscale))
    er, ed, eo = _rect_adjoints(8, 1080, 1920, (5,), RECTS_1080, 23)
    t = lambda a: torch.as_tensor(a, device="cuda")
    g = grads_to_numpy(rast.backward(gm, ct, out, dl_drgb=t(er), dl_ddepth=t(ed), dl_dopac=t(eo)))
    o = _oracle_rect_grads(oracle, m, w.cams, (5,), RECTS_1080, er, ed, eo)
    gerr = {k: rel_err(g[k], o[k]) for k in GRAD_KEYS}
    assert_grads_close(g, o, GRAD_KEYS, label=f"2M SH3 8x1080p {'BF16' if sh_bf16 else 'FP32'} SH, sampled rectangles")
    with capsys.disabled():
        print(f"\nprecision {'BF16' if sh_bf16 else 'FP32'} SH: max abs rgb {worst['rgb']:.2e} opac {worst['opac']:.2e} "
              f"depth/scale {worst['depth']:.2e}; mean abs rgb {np.mean(means['rgb']):.2e} "
              f"opac {np.mean(means['opac']):.2e}; grad rel " + " ".join(f"{k} {v:.1e}" for k, v in gerr.items()))
    assert worst["rgb"] <= IMG_TOL and worst["opac"] <= IMG_TOL and worst["depth"] <= IMG_TOL
    assert max(gerr.values()) <= GRAD_TOL
    assert rel_err(g["pose"][5], o["pose"][5]) <= GRAD_TOL


def test_tracking_32_frames_jacobian_rows_sampled(oracle):
    w = synth.tracking()
    m = host_map(w.gmap)
    rast, gm, ct, out = _render(w)
    pix = torch.as_tensor(w.meta["pix"], device="cuda")
    J, rgb = rast.pose_jacobian(gm, ct, pix)
    J, rgb = J.cpu().numpy(), rgb.cpu().numpy()
    assert J.shape == (32, 20000, 3, 6) and np.isfinite(J).all()
    rng = np.random.default_rng(4)
    for f in (0, 17):
        sel = np.sort(rng.choice(20000, 300, replace=False))
        p = w.meta["pix"][f][sel]
        Jo, rgbo = oracle.pose_jacobian(m, w.cams[f], p)
        r = oracle.render(m, w.cams[f])
        ok = r["flags"].reshape(-1)[p] == 0
        np.testing.assert_allclose(rgb[f][sel][ok], rgbo[ok], atol=IMG_TOL)
        err = np.abs(J[f][sel][ok] - Jo[ok]).max() / np.abs(Jo[ok]).max()
        assert err <= GRAD_TOL, (f, err)
    # the 6x1 gradient of an L1 photometric loss on the selected pixels equals sum_p J_p^T dL/dC_p
    f = 5
    H, W = 512, 640
    gC = np.zeros((32, 3, H, W), np.float32)
    tgt = w.tgt_rgb[f].reshape(3, -1)
    res = out.rgb[f].cpu().numpy().reshape(3, -1)[:, w.meta["pix"][f]] - tgt[:, w.meta["pix"][f]]
    dl = (np.sign(res) / (3.0 * len(w.meta["pix"][f]))).astype(np.float32)
    gC[f].reshape(3, -1)[:, w.meta["pix"][f]] = dl
    g = rast.backward(gm, ct, out, dl_drgb=torch.as_tensor(gC, device="cuda"))
    gp = g.pose.cpu().numpy()[f]
    want = np.einsum("pck,cp->k", J[f].astype(np.float64), dl.astype(np.float64))
    assert rel_err(gp, want) <= GRAD_TOL
