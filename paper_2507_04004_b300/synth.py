"""Seeded synthetic inputs shaped like the paper's mapping and tracking data.

This module only draws numbers: Gaussian maps, camera poses, LiDAR-style
sparse depth maps and target images.  It contains none of the rasterizer's
arithmetic (no projection of Gaussians, no SH evaluation, no compositing), and
both the CUDA path and the FP64 oracle take their inputs from here.

The paper's datasets (arxiv 2507.04004, Sec. "Datasets for Evaluation") are not
available, so these stand in for them:

* maps: means uniform in a box, log-scales N(-2, 0.5) per axis, uniformly
  random unit quaternions (w, x, y, z), logit opacities N(0, 1), SH DC from an
  RGB colour uniform in [0, 1] (``sh_dc = (rgb - 0.5) / Y00`` so that a degree-0
  map shows exactly that colour), higher SH coefficients N(0, 0.1);
* keyframes: pinhole cameras on a straight track along +z;
* sparse depth: a 32-ring spinning LiDAR (ring elevations evenly spread over
  [-15 deg, 15 deg], 1800 azimuth steps) cast against the walls of the map's
  box, merged over consecutive 0.1 m poses and projected into each image with
  a nearest-point z-buffer; 0 marks "no depth";
* target images: a smooth random colour field plus uniform noise.

Arrays are numpy, planar (channel-major): mean [3][N], log_scale [3][N],
quat [4][N], logit_opacity [N], sh_dc [3][N], sh_rest [K-1][3][N].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2507_04004
Y00 = 0.5 / math.sqrt(math.pi)  # constant degree-0 real SH basis value


@dataclass
class GaussianMap:
    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    logit_opacity: np.ndarray
    sh_dc: np.ndarray
    sh_rest: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.logit_opacity.shape[0])

    def as_dict(self) -> dict:
        return dict(mean=self.mean, log_scale=self.log_scale, quat=self.quat, logit_opacity=self.logit_opacity,
                    sh_dc=self.sh_dc, sh_rest=self.sh_rest, sh_degree=self.sh_degree)

    def subset(self, idx) -> "GaussianMap":
        return GaussianMap(self.mean[:, idx], self.log_scale[:, idx], self.quat[:, idx], self.logit_opacity[idx],
                           self.sh_dc[:, idx], self.sh_rest[:, :, idx], self.sh_degree)


def camera(R, t, fx, fy, cx, cy, width, height) -> dict:
    """World-to-camera pose (row-major R, t) and pinhole intrinsics."""
    return dict(R=np.asarray(R, np.float32).reshape(3, 3), t=np.asarray(t, np.float32).reshape(3),
                fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy), width=int(width), height=int(height))


def random_quaternions(rng, n) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake's method), [4][n]."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)])
    return q.astype(np.float32)


def random_map(rng, n, lo, hi, sh_degree, log_scale_mean=-2.0, log_scale_std=0.5, rest_std=0.1,
               degenerate_frac=0.0) -> GaussianMap:
    """Gaussians uniform in the box [lo, hi] (3-vectors)."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    mean = (lo[:, None] + (hi - lo)[:, None] * rng.random((3, n))).astype(np.float32)
    log_scale = rng.normal(log_scale_mean, log_scale_std, (3, n)).astype(np.float32)
    if degenerate_frac > 0:
        k = int(round(degenerate_frac * n))
        idx = rng.choice(n, size=k, replace=False)
        axis = rng.integers(0, 3, size=k)
        log_scale[axis, idx] = -8.0
    quat = random_quaternions(rng, n)
    logit = rng.normal(0.0, 1.0, n).astype(np.float32)
    rgb = rng.random((3, n))
    sh_dc = ((rgb - 0.5) / Y00).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh_rest = rng.normal(0.0, rest_std, (K - 1, 3, n)).astype(np.float32)
    return GaussianMap(mean, log_scale, quat, logit, sh_dc, sh_rest, sh_degree)


def yaw_pitch_rotation(yaw, pitch=0.0, roll=0.0) -> np.ndarray:
    """Camera-to-world rotation for a camera looking along +z (y down),
    turned by yaw about the world y axis, then pitch about x, then roll about z."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Ry = np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    Rz = np.array([[cr, -sr, 0], [sr, cr, 0], [0, 0, 1]])
    return Ry @ Rx @ Rz


def pose_from_centre(Rcw_to_world, centre) -> tuple[np.ndarray, np.ndarray]:
    """World-to-camera (R, t) of a camera with camera-to-world rotation
    ``Rcw_to_world`` placed at ``centre``."""
    R = np.asarray(Rcw_to_world, np.float64).T
    t = -R @ np.asarray(centre, np.float64)
    return R.astype(np.float32), t.astype(np.float32)


def smooth_target(rng, height, width, n_waves=6, noise=0.1) -> np.ndarray:
    """[3][H][W] colour field in [0, 1]: random sinusoids plus uniform noise."""
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float32)
    out = np.zeros((3, height, width), np.float32)
    for c in range(3):
        acc = np.full((height, width), 0.5, np.float32)
        for _ in range(n_waves):
            kx, ky = rng.normal(0, 2 * np.pi / 160.0, 2)
            ph = rng.random() * 2 * np.pi
            acc += 0.25 / math.sqrt(n_waves) * np.sin(kx * xx + ky * yy + ph).astype(np.float32)
        out[c] = acc
    out += (noise * (rng.random(out.shape) - 0.5)).astype(np.float32)
    return np.clip(out, 0.0, 1.0).astype(np.float32)


def quantize_8bit(img) -> np.ndarray:
    """The image as an 8-bit camera delivers it, in float32: round(255 c) / 255
    (an IEEE float32 division, the value the device's unpacking of the byte
    gives)."""
    k = np.round(np.clip(img, 0.0, 1.0) * 255.0).astype(np.float32)
    return (k / np.float32(255.0)).astype(np.float32)


def to_uint8(img) -> np.ndarray:
    """Bytes of an image whose values are multiples of 1/255."""
    return np.round(np.asarray(img, np.float64) * 255.0).astype(np.uint8)


def lidar_depth(cam, centre_world, Rcw, box_lo, box_hi, n_rings=32, n_az=1800, elev_deg=15.0,
                track_step=0.1, target_frac=0.03, max_scans=10) -> tuple[np.ndarray, float]:
    """Sparse depth map [H][W] (0 = none) from a spinning LiDAR at the camera.

    The scanner sits at the camera centre, ``max_scans`` consecutive scans are
    taken at 0.1 m steps backwards along the camera's viewing axis (the
    paper merges several LiDAR frames into one sparse depth map), stopping once
    ``target_frac`` of the pixels hold a depth.  Each ray ends on the first wall
    of the axis-aligned box.  Returns (depth map, fraction of valid pixels)."""
    W, H = cam["width"], cam["height"]
    Rwc = np.asarray(cam["R"], np.float64)
    tw = np.asarray(cam["t"], np.float64)
    lo, hi = np.asarray(box_lo, np.float64), np.asarray(box_hi, np.float64)
    elev = np.deg2rad(np.linspace(-elev_deg, elev_deg, n_rings))
    az = np.arange(n_az) * (2 * np.pi / n_az)
    E, A = np.meshgrid(elev, az, indexing="ij")
    # sensor frame = camera axes: x right, y down, z forward; elevation up = -y
    d_sensor = np.stack([np.cos(E) * np.sin(A), -np.sin(E), np.cos(E) * np.cos(A)], -1).reshape(-1, 3)
    d_world = d_sensor @ np.asarray(Rcw, np.float64).T
    depth = np.zeros((H, W), np.float32)
    forward = np.asarray(Rcw, np.float64)[:, 2]
    frac = 0.0
    for s in range(max_scans):
        origin = np.asarray(centre_world, np.float64) - s * track_step * forward
        with np.errstate(divide="ignore", invalid="ignore"):
            t_hi = (hi[None] - origin[None]) / d_world
            t_lo = (lo[None] - origin[None]) / d_world
        t_exit = np.where(d_world > 0, t_hi, np.where(d_world < 0, t_lo, np.inf)).min(axis=1)
        pts = origin[None] + t_exit[:, None] * d_world
        pc = pts @ Rwc.T + tw[None]
        z = pc[:, 2]
        ok = z > 0.2
        u = np.floor(cam["fx"] * pc[ok, 0] / z[ok] + cam["cx"]).astype(np.int64)
        v = np.floor(cam["fy"] * pc[ok, 1] / z[ok] + cam["cy"]).astype(np.int64)
        zz = z[ok].astype(np.float32)
        inb = (u >= 0) & (u < W) & (v >= 0) & (v < H)
        u, v, zz = u[inb], v[inb], zz[inb]
        lin = v * W + u
        order = np.argsort(-zz, kind="stable")  # far first, nearest written last wins
        flat = depth.reshape(-1)
        cur = flat[lin[order]]
        newz = zz[order]
        take = (cur == 0) | (newz < cur)
        flat[lin[order][take]] = newz[take]
        frac = float((depth > 0).mean())
        if frac >= target_frac:
            break
    return depth, frac


@dataclass
class Workload:
    name: str
    gmap: GaussianMap
    cams: list
    tgt_rgb: np.ndarray | None = None      # [V][3][H][W]
    tgt_depth: np.ndarray | None = None    # [V][H][W]
    w_rgb: float = 1.0
    w_depth: float = 0.0
    sh_bf16: bool = False
    meta: dict = field(default_factory=dict)


def tiny(seed=SEED_BASE + 1, n=2000, width=128, height=96) -> Workload:
    """2,000 Gaussians in the camera frame (identity pose), degree-0 SH,
    128x96 pinhole fx = fy = 100; uniform RGB target, 5 % depth pixels (the
    depth values themselves are filled in by the caller)."""
    rng = np.random.default_rng(seed)
    g = random_map(rng, n, (-4, -4, 2), (4, 4, 12), 0)
    cam = camera(np.eye(3), np.zeros(3), 100.0, 100.0, width / 2, height / 2, width, height)
    tgt = rng.random((1, 3, height, width)).astype(np.float32)
    mask = np.zeros((1, height, width), bool)
    k = int(round(0.05 * width * height))
    mask.reshape(-1)[rng.choice(width * height, size=k, replace=False)] = True
    noise = rng.normal(0.0, 0.05, (1, height, width)).astype(np.float32)
    return Workload("tiny", g, [cam], tgt, None, 1.0, 0.5, meta=dict(depth_mask=mask, depth_noise=noise))


def mapping(seed=SEED_BASE + 2, n=500_000, width=1280, height=720, focal=700.0, sh_degree=3, n_views=4,
            yaws=None, sh_bf16=False, degenerate_frac=0.0, w_rgb=0.8, w_depth=0.2) -> Workload:
    """Map in a 60x20x60 m box around a straight keyframe track along +z
    (0.5 m spacing); each view carries a LiDAR sparse depth map and a smooth
    random target image (8-bit, as a camera delivers it)."""
    rng = np.random.default_rng(seed)
    lo, hi = (-30.0, -10.0, -30.0), (30.0, 10.0, 30.0)
    g = random_map(rng, n, lo, hi, sh_degree, degenerate_frac=degenerate_frac)
    cams, depths, tgts, fracs = [], [], [], []
    yaws = yaws if yaws is not None else [0.0] * n_views
    for v in range(n_views):
        centre = np.array([0.0, 0.0, 0.5 * (v % 4)])
        Rc = yaw_pitch_rotation(yaws[v])
        R, t = pose_from_centre(Rc, centre)
        cam = camera(R, t, focal, focal, width / 2, height / 2, width, height)
        d, f = lidar_depth(cam, centre, Rc, lo, hi)
        cams.append(cam)
        depths.append(d)
        fracs.append(f)
        tgts.append(quantize_8bit(smooth_target(rng, height, width)))
    return Workload("mapping", g, cams, np.stack(tgts), np.stack(depths), w_rgb, w_depth, sh_bf16,
                    meta=dict(depth_frac=fracs, box=(lo, hi)))


def tracking_poses(rng, n_frames, box_lo, box_hi):
    """Ground-truth camera centres uniform in the central half of the box,
    yaw uniform, pitch N(0, 5 deg), roll 0."""
    lo, hi = np.asarray(box_lo, np.float64), np.asarray(box_hi, np.float64)
    c, r = (lo + hi) / 2, (hi - lo) / 4
    out = []
    for _ in range(n_frames):
        centre = c + r * (2 * rng.random(3) - 1)
        Rc = yaw_pitch_rotation(rng.random() * 2 * np.pi, np.deg2rad(rng.normal(0, 5.0)), 0.0)
        out.append((centre, Rc))
    return out


def pose_perturbations(rng, n_frames, rot_std=0.02, trans_std=0.05) -> np.ndarray:
    """xi = (rho, theta) per frame: rho ~ N(0, trans_std), theta ~ N(0, rot_std)."""
    xi = np.zeros((n_frames, 6))
    xi[:, :3] = rng.normal(0, trans_std, (n_frames, 3))
    xi[:, 3:] = rng.normal(0, rot_std, (n_frames, 3))
    return xi


def top_gradient_pixels(img, k) -> np.ndarray:
    """Linear indices of the k interior pixels with the largest central-difference
    gradient norm of the grey image (mean of RGB); ties go to the lower index."""
    grey = np.asarray(img, np.float64).mean(axis=0)
    H, W = grey.shape
    gx = np.zeros_like(grey)
    gy = np.zeros_like(grey)
    gx[1:-1, 1:-1] = 0.5 * (grey[1:-1, 2:] - grey[1:-1, :-2])
    gy[1:-1, 1:-1] = 0.5 * (grey[2:, 1:-1] - grey[:-2, 1:-1])
    mag = np.hypot(gx, gy)
    interior = np.zeros_like(grey, bool)
    interior[1:-1, 1:-1] = True
    lin = np.flatnonzero(interior)
    vals = mag.reshape(-1)[lin]
    order = np.lexsort((lin, -vals))
    return np.sort(lin[order[:k]]).astype(np.int32)


def se3_right_perturb(R, t, xi) -> tuple[np.ndarray, np.ndarray]:
    """World-to-camera (R, t) composed with Exp(xi) on the right, xi = (rho, theta)."""
    from scipy.linalg import expm
    X = np.zeros((4, 4))
    rho, th = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    X[:3, :3] = [[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]]
    X[:3, 3] = rho
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    Tp = T @ expm(X)
    return Tp[:3, :3].astype(np.float32), Tp[:3, 3].astype(np.float32)


def tracking(seed=SEED_BASE + 4, n=1_000_000, n_frames=32, width=640, height=512, focal=500.0, sh_degree=1,
             n_pix=20_000) -> Workload:
    """Tracking frames: a map in the 60x20x60 m box, ground-truth poses in the
    central half of the box, query poses GT Exp(xi) with theta ~ N(0, 0.02 rad)
    and rho ~ N(0, 0.05 m) per axis, smooth random targets and, per frame, the
    n_pix interior pixels with the largest target-image gradient."""
    rng = np.random.default_rng(seed)
    lo, hi = (-30.0, -10.0, -30.0), (30.0, 10.0, 30.0)
    g = random_map(rng, n, lo, hi, sh_degree)
    gt, cams, tgts, pix = [], [], [], []
    xis = pose_perturbations(rng, n_frames)
    for f, (centre, Rc) in enumerate(tracking_poses(rng, n_frames, lo, hi)):
        R, t = pose_from_centre(Rc, centre)
        gt.append(camera(R, t, focal, focal, width / 2, height / 2, width, height))
        Rq, tq = se3_right_perturb(np.asarray(R, np.float64), np.asarray(t, np.float64), xis[f])
        cams.append(camera(Rq, tq, focal, focal, width / 2, height / 2, width, height))
        img = smooth_target(rng, height, width)
        tgts.append(img)
        pix.append(top_gradient_pixels(img, n_pix))
    return Workload("tracking", g, cams, np.stack(tgts), None, 1.0, 0.0,
                    meta=dict(gt_cams=gt, xi=xis, pix=np.stack(pix)))
