"""Python face of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``oracle/liboracle.so`` (built
from ``gs_oracle.cpp`` with g++/OpenMP by :func:`build`), converts every input
to float64 and returns numpy arrays.  It imports nothing from the CUDA package.

Functions follow the paper's rasterizer (arxiv 2507.04004): projection
(Sec. "3D Gaussian Splatting Representation"), Eq. alpha, the compositing
equations rendered_rgb / rendered_depth / rendered_opacity, the tile culling
rule of Sec. "Fast Tile-based Culling", the loss of Eq. depth_loss and the
pose derivative of Eq. 3dgs_jacobi under the right perturbation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (g++ -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Map(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32),
                ("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("logit_opacity", C.c_void_p), ("sh_dc", C.c_void_p), ("sh_rest", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class _Config(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("t_min", C.c_double),
                ("near_z", C.c_double), ("dilation", C.c_double), ("fov_clamp", C.c_double),
                ("bg", C.c_double * 3)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.ocl_sh_basis.argtypes = [C.c_int32, P, P]
            lib.ocl_project.argtypes = [P, P, P] + [P] * 9
            lib.ocl_tiles.argtypes = [P, P, P, C.c_int32, C.c_double, C.c_int64, P, P, P]
            lib.ocl_tiles.restype = C.c_int64
            lib.ocl_render.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_double] + [P] * 7
            lib.ocl_backward.argtypes = ([P, C.c_int32, P, P, P, P, C.c_double, C.c_double, P, P, P]
                                         + [C.c_int32] * 4 + [P] * 8)
            lib.ocl_pose_jacobian.argtypes = [P, P, P, P, C.c_int32, P, P]
            lib.ocl_depth_keys.argtypes = [P, P, P]
            lib.ocl_set_threads.argtypes = [C.c_int32]
            lib.ocl_get_threads.restype = C.c_int32
            _lib = lib
    return _lib


DEFAULT_CONFIG = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, near_z=0.2, dilation=0.3,
                      fov_clamp=1.3, bg=(0.0, 0.0, 0.0))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _MapHandle:
    """Keeps the float64 copies alive while the C struct points at them."""

    def __init__(self, m):
        self.arrays = {k: _f64(m[k]) for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc")}
        deg = int(m["sh_degree"])
        rest = m.get("sh_rest")
        if deg > 0:
            self.arrays["sh_rest"] = _f64(rest)
        n = self.arrays["logit_opacity"].shape[-1]
        self.n = n
        self.deg = deg
        self.s = _Map(n, deg, *(self.arrays[k].ctypes.data for k in
                                ("mean", "log_scale", "quat", "logit_opacity", "sh_dc")),
                      self.arrays["sh_rest"].ctypes.data if deg > 0 else None)


def _cam(c):
    s = _Camera()
    R = np.asarray(c["R"], dtype=np.float64).reshape(9)
    t = np.asarray(c["t"], dtype=np.float64).reshape(3)
    for i in range(9):
        s.R[i] = R[i]
    for i in range(3):
        s.t[i] = t[i]
    s.fx, s.fy, s.cx, s.cy = (float(c[k]) for k in ("fx", "fy", "cx", "cy"))
    s.width, s.height = int(c["width"]), int(c["height"])
    return s


def _cfg(cfg=None):
    d = dict(DEFAULT_CONFIG)
    if cfg:
        d.update(cfg)
    s = _Config()
    for k in ("alpha_min", "alpha_max", "t_min", "near_z", "dilation", "fov_clamp"):
        setattr(s, k, float(d[k]))
    for i in range(3):
        s.bg[i] = float(d["bg"][i])
    return s


def _p(a):
    return None if a is None else a.ctypes.data


def sh_basis(deg: int, direction) -> np.ndarray:
    """Real SH basis values (16 slots, zero beyond degree ``deg``)."""
    lib = _load()
    d = _f64(direction).reshape(3)
    Y = np.zeros(16)
    lib.ocl_sh_basis(int(deg), _p(d), _p(Y))
    return Y


def depth_keys(m, cam) -> np.ndarray:
    lib = _load()
    mh = _MapHandle(m)
    keys = np.zeros(mh.n, dtype=np.float32)
    c = _cam(cam)
    lib.ocl_depth_keys(C.byref(mh.s), C.byref(c), _p(keys))
    return keys


def project(m, cam, cfg=None) -> dict:
    """Per-Gaussian projection of one view (planar arrays [c][n])."""
    lib = _load()
    mh = _MapHandle(m)
    n = mh.n
    out = dict(valid=np.zeros(n, np.int32), mean2d=np.zeros((2, n)), cov2d=np.zeros((3, n)),
               conic=np.zeros((3, n)), opacity=np.zeros(n), rgb=np.zeros((3, n)), depth=np.zeros(n),
               depth32=np.zeros(n, np.float32), clamp_flags=np.zeros(n, np.int32))
    c, k = _cam(cam), _cfg(cfg)
    lib.ocl_project(C.byref(mh.s), C.byref(c), C.byref(k), *(_p(out[x]) for x in (
        "valid", "mean2d", "cov2d", "conic", "opacity", "rgb", "depth", "depth32", "clamp_flags")))
    return out


def tiles(m, cam, cfg=None, brute=False, margin_eps=1e-4):
    """Sorted (tile, gid, margin) pairs of one view; margin 0 = clean pass,
    1 = pass near the threshold, 2 = fail near the threshold."""
    lib = _load()
    mh = _MapHandle(m)
    c, k = _cam(cam), _cfg(cfg)
    cap = 1 << 16
    while True:
        tile = np.zeros(cap, np.int32)
        gid = np.zeros(cap, np.int32)
        margin = np.zeros(cap, np.int32)
        npairs = lib.ocl_tiles(C.byref(mh.s), C.byref(c), C.byref(k), int(bool(brute)), float(margin_eps),
                               cap, _p(tile), _p(gid), _p(margin))
        if npairs >= 0:
            return tile[:npairs], gid[:npairs], margin[:npairs]
        cap = -npairs


def render(m, cam, cfg=None, rect=None, brute=False, margin_eps=1e-4) -> dict:
    """Render a pixel rectangle (x0, y0, w, h) of one view (default: all)."""
    lib = _load()
    mh = _MapHandle(m)
    c, k = _cam(cam), _cfg(cfg)
    x0, y0, w, h = rect if rect is not None else (0, 0, c.width, c.height)
    out = dict(rgb=np.zeros((3, h, w)), depth=np.zeros((h, w)), opac=np.zeros((h, w)),
               t_final=np.zeros((h, w)), n_contrib=np.zeros((h, w), np.int32),
               last_gid=np.zeros((h, w), np.int32), flags=np.zeros((h, w), np.int32))
    lib.ocl_render(C.byref(mh.s), C.byref(c), C.byref(k), x0, y0, w, h, int(bool(brute)), float(margin_eps),
                   *(_p(out[x]) for x in ("rgb", "depth", "opac", "t_final", "n_contrib", "last_gid", "flags")))
    return out


def backward(m, cams, cfg=None, tgt_rgb=None, tgt_depth=None, w_rgb=1.0, w_depth=0.0,
             ext_rgb=None, ext_depth=None, ext_opac=None, rect=None) -> dict:
    """Loss and gradients over a list of views.

    With ``tgt_rgb`` the fused loss of Eq. depth_loss is used (L1 colour mean
    over 3HW weighted by ``w_rgb`` plus opacity-normalised L1 depth over the
    valid LiDAR pixels weighted by ``w_depth``, summed over views); otherwise
    the pixel adjoints ``ext_*`` ([V][3][H][W], [V][H][W]) are back-propagated.
    ``rect`` restricts the back-propagated pixels (normalisers stay global)."""
    lib = _load()
    mh = _MapHandle(m)
    V = len(cams)
    cs = (_Camera * V)(*[_cam(x) for x in cams])
    k = _cfg(cfg)
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    x0, y0, w, h = rect if rect is not None else (0, 0, W, H)
    n, deg = mh.n, mh.deg
    K = (deg + 1) ** 2
    tr = None if tgt_rgb is None else _f64(tgt_rgb)
    td = None if tgt_depth is None else _f64(tgt_depth)
    er = None if ext_rgb is None else _f64(ext_rgb)
    ed = None if ext_depth is None else _f64(ext_depth)
    eo = None if ext_opac is None else _f64(ext_opac)
    out = dict(loss=np.zeros(V), mean=np.zeros((3, n)), log_scale=np.zeros((3, n)), quat=np.zeros((4, n)),
               logit_opacity=np.zeros(n), sh_dc=np.zeros((3, n)),
               sh_rest=np.zeros((max(K - 1, 1), 3, n)), pose=np.zeros((V, 6)))
    lib.ocl_backward(C.byref(mh.s), V, cs, C.byref(k), _p(tr), _p(td), float(w_rgb), float(w_depth),
                     _p(er), _p(ed), _p(eo), x0, y0, w, h,
                     *(_p(out[x]) for x in ("loss", "mean", "log_scale", "quat", "logit_opacity", "sh_dc",
                                            "sh_rest", "pose")))
    if K == 1:
        out["sh_rest"] = np.zeros((0, 3, n))
    return out


def pose_jacobian(m, cam, pix, cfg=None):
    """J [n_pix][3][6] = dC/dxi (right perturbation, xi = (rho, theta)) and
    the rendered colour [n_pix][3] at the listed linear pixel indices."""
    lib = _load()
    mh = _MapHandle(m)
    c, k = _cam(cam), _cfg(cfg)
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32))
    J = np.zeros((len(pix), 3, 6))
    rgb = np.zeros((len(pix), 3))
    lib.ocl_pose_jacobian(C.byref(mh.s), C.byref(c), C.byref(k), _p(pix), len(pix), _p(J), _p(rgb))
    return J, rgb


def set_threads(n: int) -> None:
    """Number of threads the oracle's parallel loops use from now on."""
    _load().ocl_set_threads(int(n))


def threads() -> int:
    return int(_load().ocl_get_threads())
