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


# Lines gathered by the parity tests (pair counts, element-wise gradient
# errors); conftest prints them in pytest's terminal summary.
REPORT: list = []


def report(line: str) -> None:
    REPORT.append(line)


def gpu_tile_pairs(rast, view):
    """(tile, gid) pairs of one view in sorted order, from the workspace."""
    start, count, ids = (t.cpu().numpy() for t in rast.tile_lists())
    T = ((rast.width + 15) // 16) * ((rast.height + 15) // 16)
    c = count[view * T:(view + 1) * T].astype(np.int64)
    s = start[view * T:(view + 1) * T].astype(np.int64)
    tiles = np.repeat(np.arange(T, dtype=np.int32), c)
    # positions of every tile's pairs, tile after tile
    pos = np.repeat(s - np.concatenate([[0], np.cumsum(c)[:-1]]), c) + np.arange(int(c.sum()), dtype=np.int64)
    return tiles, ids[pos]


def compare_tiles(oracle, m, cam, rast, view, label=None, cfg=None):
    """Bit-exact tile lists / order outside the oracle's threshold margin:
    every pair the oracle marks as within 1e-4 (relative, in q) of the
    culling threshold is left out on both sides, everything else must match
    in content and order.  Returns the number of margin pairs seen.  cfg: the
    rasterizer constants both sides use (the oracle's defaults when None)."""
    ot, og, om = oracle.tiles(m, cam) if cfg is None else oracle.tiles(m, cam, cfg=cfg)
    gt, gg = gpu_tile_pairs(rast, view)
    n = np.int64(max(int(m["logit_opacity"].shape[0]), 1))
    code = lambda t, g: t.astype(np.int64) * n + g.astype(np.int64)
    margin_codes = code(ot[om != 0], og[om != 0])
    keep_o = om == 0
    keep_g = ~np.isin(code(gt, gg), margin_codes)
    np.testing.assert_array_equal(gt[keep_g], ot[keep_o])
    np.testing.assert_array_equal(gg[keep_g], og[keep_o])
    if label is not None:
        report(f"tile lists {label}: {int(keep_o.sum())} pairs bit-exact in content and order, "
               f"{int((om == 1).sum())} + {int((om == 2).sum())} pairs within the threshold margin "
               f"(oracle pass / fail), GPU lists {len(gt)} pairs")
    return int(len(margin_codes))


def rel_err(a, b, eps=1e-6):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), eps))


def elementwise_err(a, b, floor=1e-3):
    """Largest element-wise relative error |a - b| / (|b| + floor * max|b|)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    if b.size == 0:
        return 0.0
    scale = max(float(np.abs(b).max()), 1e-30)
    return float((np.abs(a - b) / (np.abs(b) + floor * scale)).max())


def assert_grads_close(g_gpu, g_or, keys, tol=GRAD_TOL, label=None):
    """Inf-norm relative error per parameter block <= tol; with a label, both
    it and the element-wise error go to the parity report."""
    parts = []
    for k in keys:
        a, b = np.asarray(g_gpu[k], np.float64), np.asarray(g_or[k], np.float64)
        if b.size == 0:
            continue
        e = rel_err(a, b)
        parts.append(f"{k} {e:.1e}/{elementwise_err(a, b):.1e}")
        assert e <= tol, f"{k}: relative error {e:.3e} > {tol}"
    if label is not None:
        report(f"gradients {label} (inf-norm / element-wise rel. error): " + ", ".join(parts))


def grads_to_numpy(g):
    return dict(mean=g.mean.cpu().numpy(), log_scale=g.log_scale.cpu().numpy(), quat=g.quat.cpu().numpy(),
                logit_opacity=g.logit_opacity.cpu().numpy(), sh_dc=g.sh_dc.cpu().numpy(),
                sh_rest=g.sh_rest.cpu().numpy(), pose=g.pose.cpu().numpy(), loss=g.loss.cpu().numpy())
