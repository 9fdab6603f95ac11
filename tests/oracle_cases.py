"""Small hand-built scenes for pinning the oracle (no oracle arithmetic here)."""
import math

import numpy as np

from paper_2507_04004_b300 import synth


def one_gaussian_map(means, log_scales, logits, rgbs, quats=None):
    """Degree-0 map from explicit per-Gaussian values (lists of equal length)."""
    n = len(means)
    mean = np.asarray(means, np.float64).T.copy()
    ls = np.asarray(log_scales, np.float64)
    log_scale = (np.repeat(ls[None], 3, 0) if ls.ndim == 1 else ls.T).copy()
    quat = np.asarray(quats, np.float64).T.copy() if quats is not None else np.tile([[1.0], [0], [0], [0]], (1, n))
    logit = np.asarray(logits, np.float64)
    sh_dc = ((np.asarray(rgbs, np.float64) - 0.5) / synth.Y00).T.copy()
    return dict(mean=mean, log_scale=log_scale, quat=quat, logit_opacity=logit, sh_dc=sh_dc,
                sh_rest=np.zeros((0, 3, n)), sh_degree=0)


def identity_camera(width=64, height=48, f=50.0):
    return synth.camera(np.eye(3), np.zeros(3), f, f, width / 2, height / 2, width, height)


def logit(p):
    return math.log(p / (1 - p))


def small_scene(seed=7, n=600, width=80, height=56, focal=60.0, sh_degree=3):
    """A random map seen from inside a box (degree-3 SH) for FD checks."""
    rng = np.random.default_rng(seed)
    g = synth.random_map(rng, n, (-3, -2, 1), (3, 2, 9), sh_degree, log_scale_mean=-1.5)
    R = synth.yaw_pitch_rotation(0.1, -0.05, 0.02)
    Rw, t = synth.pose_from_centre(R, (0.1, -0.2, -0.3))
    cam = synth.camera(Rw, t, focal, focal * 1.05, width / 2 + 1.5, height / 2 - 2.0, width, height)
    return g.as_dict(), cam
