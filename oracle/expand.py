"""FP64 reference of the point selection of map expansion (test
infrastructure only).

Sec. "Expansion of Gaussian Map": render the opacity map O of the new
keyframe (Eq. rendered_opacity), form the mask O < tau, and initialise new
Gaussians only from the 3D points that project into the masked pixels.  A
point p (world frame) with camera-frame position q = R p + t is selected iff
q_z > near, its pixel (floor(fx q_x / q_z + cx), floor(fy q_y / q_z + cy))
lies in the image (pixel i covers [i, i + 1), its centre is i + 0.5), and O
there is below tau.  The selected indices keep the input order.
"""
from __future__ import annotations

import numpy as np


def select_points(points, cam, opac, tau=0.99, near=0.2):
    """points [3][P] (world), cam: camera dict, opac [H][W]: indices of the
    selected points (ascending) and, per point, the distance in pixels of its
    projection to the nearest pixel border (for callers that compare with an
    FP32 implementation)."""
    p = np.asarray(points, np.float64)
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], np.float64).reshape(3, 1)
    q = R @ p + t
    z = q[2]
    front = z > near
    zs = np.where(front, z, 1.0)
    u = cam["fx"] * q[0] / zs + cam["cx"]
    v = cam["fy"] * q[1] / zs + cam["cy"]
    H, W = opac.shape
    i, j = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
    inside = front & (i >= 0) & (i < W) & (j >= 0) & (j < H)
    o = np.where(inside, opac[np.clip(j, 0, H - 1), np.clip(i, 0, W - 1)], np.inf)
    sel = inside & (o < tau)
    border = np.minimum(np.minimum(u - np.floor(u), np.ceil(u) - u), np.minimum(v - np.floor(v), np.ceil(v) - v))
    return np.nonzero(sel)[0], border
