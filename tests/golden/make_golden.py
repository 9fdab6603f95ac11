"""Writes tests/golden/tiny3.json, a regression fixture for the oracle and a
fixed target for the CUDA path.

The scene is built by hand: three overlapping Gaussians at different depths
(one nearly opaque, so that alpha is clamped at 0.99; one elongated and
rotated), SH degree 1, seen by a slightly rotated camera of 24 x 20 pixels (two
tiles across and two down, both ragged). The expected values are the FP64
oracle's image (Eq. alpha, Eq. rendered_rgb, rendered_depth, rendered_opacity),
each pixel's number of blended Gaussians and last blended Gaussian, its
per-pixel decision flags, and the loss and gradients of the fused loss of
Eq. depth_loss (0.8 L1 colour + 0.2 opacity-normalised L1 depth on four LiDAR
pixels), including the pose gradient of Eq. 3dgs_jacobi.

These values come from the oracle, so they are not a pin of it (the pins are
the closed forms, brute force and finite differences of the oracle tests):
they record the oracle's output so that a change to its arithmetic shows, and
give the GPU tests a stored target.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny3.json")


def scene():
    """Parameters, camera and targets of the fixture (plain numbers)."""
    W, H = 24, 20
    c, s = np.cos(0.08), np.sin(0.08)
    R = [[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]]       # camera rotated 0.08 rad about y
    cam = dict(R=R, t=[0.05, -0.03, 0.1], fx=22.0, fy=21.0, cx=11.5, cy=10.25, width=W, height=H)
    m = dict(
        mean=[[-0.30, 0.25, 0.05], [0.10, -0.20, 0.30], [3.0, 3.6, 4.2]],   # [3][n]: x, y, z rows
        log_scale=[[-1.2, -0.9, -1.5], [-1.1, -2.2, -1.4], [-1.3, -1.0, -1.6]],
        quat=[[1.0, 0.9, 0.8], [0.0, 0.3, -0.2], [0.0, -0.2, 0.4], [0.0, 0.25, 0.1]],
        logit_opacity=[6.5, 0.4, -0.3],                        # sigmoid(6.5) = 0.9985: alpha clamped
        sh_dc=[[0.8, -0.4, 0.1], [-0.2, 0.6, 0.3], [0.1, 0.2, -0.7]],
        sh_rest=[[[0.10, -0.05, 0.02], [0.03, 0.08, -0.04], [-0.06, 0.01, 0.05]],
                 [[0.02, 0.04, -0.03], [-0.05, 0.02, 0.06], [0.07, -0.02, 0.01]],
                 [[-0.04, 0.03, 0.08], [0.01, -0.06, 0.02], [0.03, 0.05, -0.01]]],
        sh_degree=1)
    yy, xx = np.mgrid[0:H, 0:W]
    tgt_rgb = np.stack([0.3 + 0.4 * ((xx // 3 + yy // 3) % 2), 0.2 + 0.02 * xx, 0.7 - 0.025 * yy])[None]
    tgt_depth = np.zeros((1, H, W))
    for (y, x, d) in ((4, 5, 3.1), (9, 12, 3.7), (12, 8, 4.0), (15, 18, 4.4)):
        tgt_depth[0, y, x] = d
    return m, cam, tgt_rgb, tgt_depth


def host(m):
    return {k: (np.asarray(v, np.float32) if isinstance(v, list) else v) for k, v in m.items()}


def compute():
    m, cam, tgt_rgb, tgt_depth = scene()
    hm = host(m)
    tr, td = tgt_rgb.astype(np.float32), tgt_depth.astype(np.float32)
    r = O.render(hm, cam)
    b = O.backward(hm, [cam], tgt_rgb=tr, tgt_depth=td, w_rgb=0.8, w_depth=0.2)
    return dict(rgb=r["rgb"], depth=r["depth"], opac=r["opac"], t_final=r["t_final"], n_contrib=r["n_contrib"],
                last_gid=r["last_gid"], flags=r["flags"], loss=b["loss"], grad_mean=b["mean"], grad_log_scale=b["log_scale"],
                grad_quat=b["quat"], grad_logit_opacity=b["logit_opacity"], grad_sh_dc=b["sh_dc"],
                grad_sh_rest=b["sh_rest"], grad_pose=b["pose"])


def main():
    O.build()
    m, cam, tgt_rgb, tgt_depth = scene()
    exp = compute()
    doc = {"about": "FP64 oracle output for the hand-built three-Gaussian scene of make_golden.py "
                    "(Eq. alpha, rendered_rgb/depth/opacity, depth_loss, 3dgs_jacobi); a regression fixture, "
                    "not a pin",
           "expected": {k: np.asarray(v).tolist() for k, v in exp.items()}}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
