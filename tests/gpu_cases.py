"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on a
workload from ``synth`` and compare with the oracle on the same inputs."""
import numpy as np
import torch

from paper_2507_04004_b300 import synth

IMG_TOL = 1e-4      # max abs error of RGB and O (FP32 path vs FP64 oracle)
GRAD_TOL = 1e-3     # relative (inf-norm per parameter block) gradient error


def host_map(g: synth.GaussianMap, sh_bf16=False) -> dict:
    """The map as the oracle must see it: BF16 SH rounded exactly as the GPU reads it."""
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.as_dict().items()}
    if sh_bf16:
        for k in ("sh_dc", "sh_rest"):
            d[k] = torch.as_tensor(d[k]).to(torch.bfloat16).to(torch.float32).numpy()
    return d


def gpu_render(g, cams, sh_bf16=False, capacity=None, config=None, backward="pixel"):
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    gm = GaussianMap.from_host(g, sh_bf16=sh_bf16)
    W, H = cams[0]["width"], cams[0]["height"]
    rast = Rasterizer(gm.n, len(cams), W, H, pair_capacity=capacity, config=config, backward=backward)
    ct = cameras_tensor(cams)
    out = rast.render(gm, ct)
    torch.cuda.synchronize()
    return rast, gm, ct, out


def gpu_tile_pairs(rast, view):
    """(tile, gid) pairs of one view in sorted order, from the workspace."""
    start, count, ids = (t.cpu().numpy() for t in rast.tile_lists())
    T = ((rast.width + 15) // 16) * ((rast.height + 15) // 16)
    tiles, gids = [], []
    for t in range(T):
        s, c = start[view * T + t], count[view * T + t]
        tiles.append(np.full(c, t, np.int32))
        gids.append(ids[s:s + c])
    return np.concatenate(tiles), np.concatenate(gids)


def compare_tiles(oracle, m, cam, rast, view):
    """Bit-exact tile lists / order outside the oracle's threshold margin.
    Returns the number of margin pairs seen."""
    ot, og, om = oracle.tiles(m, cam)
    gt, gg = gpu_tile_pairs(rast, view)
    margin = set(zip(ot[om != 0].tolist(), og[om != 0].tolist()))
    keep_o = om == 0
    keep_g = np.array([(a, b) not in margin for a, b in zip(gt.tolist(), gg.tolist())], bool) if len(gt) else \
        np.zeros(0, bool)
    np.testing.assert_array_equal(gt[keep_g], ot[keep_o])
    np.testing.assert_array_equal(gg[keep_g], og[keep_o])
    return len(margin)


def rel_err(a, b, eps=1e-6):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), eps))


def assert_grads_close(g_gpu, g_or, keys, tol=GRAD_TOL):
    for k in keys:
        a, b = np.asarray(g_gpu[k], np.float64), np.asarray(g_or[k], np.float64)
        if b.size == 0:
            continue
        e = rel_err(a, b)
        assert e <= tol, f"{k}: relative error {e:.3e} > {tol}"


def grads_to_numpy(g):
    return dict(mean=g.mean.cpu().numpy(), log_scale=g.log_scale.cpu().numpy(), quat=g.quat.cpu().numpy(),
                logit_opacity=g.logit_opacity.cpu().numpy(), sh_dc=g.sh_dc.cpu().numpy(),
                sh_rest=g.sh_rest.cpu().numpy(), pose=g.pose.cpu().numpy(), loss=g.loss.cpu().numpy())
