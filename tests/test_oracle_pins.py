"""Pins of the FP64 oracle to facts other than itself.

Each test checks the oracle against a closed form, a library routine, brute
force, an invariant the method guarantees, or central finite differences of
its own (separately pinned) forward pass.  References are to arxiv 2507.04004.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.special import sph_harm_y

from paper_2507_04004_b300 import synth
from tests.oracle_cases import identity_camera, logit, one_gaussian_map, small_scene

A_MIN = 1.0 / 255.0


# ---------------------------------------------------------------- SH basis
def test_sh_basis_matches_scipy_complex_harmonics(oracle):
    """Real SH with Condon-Shortley phase = sqrt2 Re/Im of scipy's complex Y_l^m
    (the view-dependent colour of Sec. 3DGS representation)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                ref = sph_harm_y(l, abs(m), theta, phi)
                if m > 0:
                    want = math.sqrt(2) * ref.real
                elif m < 0:
                    want = math.sqrt(2) * ref.imag
                else:
                    want = ref.real
                assert Y[l * l + l + m] == pytest.approx(want, abs=1e-12), (l, m)


def test_sh_basis_orthonormal_by_quadrature(oracle):
    """Gauss-Legendre x uniform-azimuth quadrature of Y_i Y_j over the sphere is I."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, wz in zip(xg, wg):
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            s = math.sqrt(1 - z * z)
            Y = oracle.sh_basis(3, [s * math.cos(phi), s * math.sin(phi), z])
            G += wz * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree_one_closed_form(oracle):
    """Y_1^{-1,0,1} = sqrt(3/4pi) * (-y, z, -x) (Condon-Shortley phase)."""
    d = np.array([0.48, -0.6, 0.64])
    Y = oracle.sh_basis(1, d)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:4], [0.5 / math.sqrt(math.pi), -c1 * d[1], c1 * d[2], -c1 * d[0]], atol=1e-15)
    assert np.all(Y[4:] == 0)


# ---------------------------------------------------------------- projection
def test_projection_isotropic_on_axis_closed_form(oracle):
    """mu' = (cx, cy) and Sigma' = (f s / d)^2 I + 0.3 I for an isotropic
    Gaussian on the optical axis, identity pose."""
    cam = identity_camera(64, 48, 50.0)
    m = one_gaussian_map([[0, 0, 5.0]], [math.log(0.2)], [logit(0.8)], [[0.2, 0.5, 0.9]])
    p = oracle.project(m, cam)
    assert p["valid"][0] == 1
    np.testing.assert_allclose(p["mean2d"][:, 0], [32.0, 24.0], atol=1e-12)
    s2 = (50 * 0.2 / 5.0) ** 2
    np.testing.assert_allclose(p["cov2d"][:, 0], [s2 + 0.3, 0.0, s2 + 0.3], atol=1e-12)
    np.testing.assert_allclose(p["conic"][:, 0], [1 / (s2 + 0.3), 0.0, 1 / (s2 + 0.3)], atol=1e-12)
    assert p["opacity"][0] == pytest.approx(0.8, abs=1e-12)
    np.testing.assert_allclose(p["rgb"][:, 0], [0.2, 0.5, 0.9], atol=1e-12)
    assert p["depth"][0] == pytest.approx(5.0, abs=1e-12)


def test_projection_rotated_anisotropic_closed_form(oracle):
    """A Gaussian rotated by phi about the optical axis projects to
    (f/d)^2 R2(phi) diag(sx^2, sy^2) R2^T + 0.3 I (quaternion (cos phi/2, 0, 0, sin phi/2))."""
    cam = identity_camera(64, 48, 40.0)
    phi, sx, sy, sz, d = 0.7, 0.3, 0.1, 0.05, 4.0
    q = [math.cos(phi / 2), 0, 0, math.sin(phi / 2)]
    m = one_gaussian_map([[0, 0, d]], [[math.log(sx), math.log(sy), math.log(sz)]], [0.0], [[0.5] * 3], [q])
    p = oracle.project(m, cam)
    R2 = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    S = (40.0 / d) ** 2 * R2 @ np.diag([sx ** 2, sy ** 2]) @ R2.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][:, 0], [S[0, 0], S[0, 1], S[1, 1]], atol=1e-12)


def test_projection_off_axis_jacobian_and_fov_clamp(oracle):
    """Off-axis isotropic Gaussian: J = [[f/z, 0, -f x/z^2], [0, f/z, 0]], and
    x/z clamped to 1.3 * W / (2 f) inside J only (mu' is not clamped)."""
    f, W, H = 40.0, 64, 48
    cam = identity_camera(W, H, f)
    s = 0.2
    for x, z in ((1.0, 4.0), (9.0, 4.0)):
        m = one_gaussian_map([[x, 0, z]], [math.log(s)], [0.0], [[0.5] * 3])
        p = oracle.project(m, cam)
        tx = min(x / z, 1.3 * W / (2 * f))
        J = np.array([[f / z, 0, -f * tx / z], [0, f / z, 0]])
        S = s * s * J @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(p["cov2d"][:, 0], [S[0, 0], S[0, 1], S[1, 1]], atol=1e-12)
        assert p["mean2d"][0, 0] == pytest.approx(f * x / z + W / 2, abs=1e-12)
        assert p["clamp_flags"][0] & 1 == (1 if x / z > 1.3 * W / (2 * f) else 0)


def test_near_plane_cut_uses_depth_key(oracle):
    cam = identity_camera()
    m = one_gaussian_map([[0, 0, 0.19], [0, 0, 0.21]], [math.log(0.01)] * 2, [0.0] * 2, [[0.5] * 3] * 2)
    assert list(oracle.project(m, cam)["valid"]) == [0, 1]


def test_view_dependent_colour_degree_one(oracle):
    """Colour = 0.5 + SH_00 Y00 + k Y_1^0(dir), dir from the camera centre
    c_w = -R^T t to the mean (camera translated to z = -1)."""
    cam = synth.camera(np.eye(3), [0, 0, 1.0], 50, 50, 32, 24, 64, 48)
    m = one_gaussian_map([[1.0, 0, 3.0]], [math.log(0.1)], [0.0], [[0.4, 0.5, 0.6]])
    m["sh_degree"] = 1
    m["sh_rest"] = np.zeros((3, 3, 1))
    m["sh_rest"][1, :, 0] = [0.3, -0.2, 0.1]  # the m = 0 (z) coefficient
    p = oracle.project(m, cam)
    d = np.array([1.0, 0, 4.0]) / math.sqrt(17.0)
    want = np.array([0.4, 0.5, 0.6]) + np.array([0.3, -0.2, 0.1]) * math.sqrt(3 / (4 * math.pi)) * d[2]
    np.testing.assert_allclose(p["rgb"][:, 0], want, atol=1e-12)


# ---------------------------------------------------------------- compositing
def _alpha_single(cam, mx, my, var, o):
    """o exp(-q/2) at every pixel centre for an isotropic 2D Gaussian."""
    yy, xx = np.mgrid[0:cam["height"], 0:cam["width"]] + 0.5
    q = ((xx - mx) ** 2 + (yy - my) ** 2) / var
    return o * np.exp(-0.5 * q)


def _alpha_proj(cam, p, i, o):
    """o exp(-q/2) at every pixel centre from a projected mean and conic."""
    yy, xx = np.mgrid[0:cam["height"], 0:cam["width"]] + 0.5
    dx, dy = xx - p["mean2d"][0, i], yy - p["mean2d"][1, i]
    a, b, c = p["conic"][:, i]
    return o * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))


def test_single_gaussian_image_closed_form(oracle):
    """C = c alpha, D = d alpha, O = alpha with alpha = min(0.99, o e^{-q/2}) or
    0 below 1/255 (Eq. alpha and Eq. rendered_rgb/depth/opacity, one term)."""
    cam = identity_camera(64, 48, 50.0)
    rgb = [0.2, 0.5, 0.9]
    for o, s in ((0.8, 0.2), (0.999, 0.65)):
        m = one_gaussian_map([[0, 0, 5.0]], [math.log(s)], [logit(o)], [rgb])
        r = oracle.render(m, cam)
        a = _alpha_single(cam, 32.0, 24.0, (50 * s / 5.0) ** 2 + 0.3, o)
        a = np.where(a >= A_MIN, np.minimum(a, 0.99), 0.0)
        for c in range(3):
            np.testing.assert_allclose(r["rgb"][c], rgb[c] * a, atol=1e-12)
        np.testing.assert_allclose(r["depth"], 5.0 * a, atol=1e-12)
        np.testing.assert_allclose(r["opac"], a, atol=1e-12)
        np.testing.assert_allclose(r["t_final"], 1 - a, atol=1e-12)
        assert (r["n_contrib"] == (a > 0)).all()
    assert r["opac"].max() == pytest.approx(0.99)  # clamp reached for o = 0.999


def test_single_gaussian_tile_list_is_the_disc(oracle):
    """Tiles kept = tiles holding a pixel centre inside q <= 2 ln(255 o)
    (Sec. Fast Tile-based Culling, exact discrete maximum)."""
    cam = identity_camera(96, 80, 50.0)
    o = 0.6
    m = one_gaussian_map([[0.31, -0.17, 5.0]], [math.log(0.25)], [logit(o)], [[0.5] * 3])
    p = oracle.project(m, cam)
    mx, my = p["mean2d"][:, 0]
    a = _alpha_single(cam, mx, my, p["cov2d"][0, 0], o)
    want = set()
    for ty in range(0, 80, 16):
        for tx in range(0, 96, 16):
            if (a[ty:ty + 16, tx:tx + 16] >= A_MIN).any():
                want.add((ty // 16) * 6 + tx // 16)
    tile, gid, margin = oracle.tiles(m, cam)
    assert set(tile[margin != 2].tolist()) == want
    assert (gid == 0).all()


def test_two_gaussians_front_to_back(oracle):
    """C = c1 a1 + c2 a2 (1 - a1) with 1 the nearer Gaussian, whatever the
    index order; equal depths fall back to index order."""
    cam = identity_camera(48, 40, 40.0)
    c1, c2 = [0.9, 0.1, 0.2], [0.1, 0.8, 0.3]
    for order in ((0, 1), (1, 0)):
        means = [[0.0, 0, 4.0], [0.0, 0.0, 6.0]]
        scales = [math.log(0.15), math.log(0.15 * 1.2)]
        ops, cols = [0.7, 0.6], [c1, c2]
        idx = list(order)
        m = one_gaussian_map([means[i] for i in idx], [scales[i] for i in idx], [logit(ops[i]) for i in idx],
                             [cols[i] for i in idx])
        r = oracle.render(m, cam)
        near, far = idx.index(0), idx.index(1)
        a1 = _alpha_single(cam, 24.0, 20.0, (40 * 0.15 / 4.0) ** 2 + 0.3, ops[0])
        a2 = _alpha_single(cam, 24.0, 20.0, (40 * 0.18 / 6.0) ** 2 + 0.3, ops[1])
        a1 = np.where(a1 >= A_MIN, np.minimum(a1, 0.99), 0)
        a2 = np.where(a2 >= A_MIN, np.minimum(a2, 0.99), 0)
        for c in range(3):
            np.testing.assert_allclose(r["rgb"][c], c1[c] * a1 + c2[c] * a2 * (1 - a1), atol=1e-12)
        np.testing.assert_allclose(r["depth"], 4.0 * a1 + 6.0 * a2 * (1 - a1), atol=1e-12)
        assert near != far
    # equal depth keys: the lower index is blended first
    m = one_gaussian_map([[0.05, 0, 5.0], [-0.05, 0, 5.0]], [math.log(0.2)] * 2, [logit(0.7), logit(0.5)], [c1, c2])
    r = oracle.render(m, cam)
    p = oracle.project(m, cam)
    assert p["depth32"][0] == p["depth32"][1]
    a0 = _alpha_proj(cam, p, 0, 0.7)
    a1 = _alpha_proj(cam, p, 1, 0.5)
    a0 = np.where(a0 >= A_MIN, np.minimum(a0, 0.99), 0)
    a1 = np.where(a1 >= A_MIN, np.minimum(a1, 0.99), 0)
    np.testing.assert_allclose(r["rgb"][0], c1[0] * a0 + c2[0] * a1 * (1 - a0), atol=1e-12)


def test_transmittance_stop_rule(oracle):
    """Identical-footprint layers of weight a: the k-th layer is blended only
    while (1-a)^k >= 1e-4 (compositing stops before the layer that would drop
    T below the cutoff)."""
    cam = identity_camera(32, 32, 40.0)
    d0, s0, o = 3.0, 0.3, 0.55
    depths = [d0 + 0.1 * k for k in range(30)]
    m = one_gaussian_map([[0, 0, d] for d in depths], [math.log(s0 * d / d0) for d in depths],
                         [logit(o)] * 30, [[0.5] * 3] * 30)
    r = oracle.render(m, cam)
    a = _alpha_single(cam, 16.0, 16.0, (40.0 * s0 / d0) ** 2 + 0.3, o)[16, 16]
    k = 0
    while (1 - a) ** (k + 1) >= 1e-4:
        k += 1
    assert r["n_contrib"][16, 16] == k
    assert r["t_final"][16, 16] == pytest.approx((1 - a) ** k, rel=1e-12)
    assert r["last_gid"][16, 16] == k - 1


def test_invariants_random_scene(oracle):
    """T_final >= 1e-4, O = 1 - T_final, 0 <= C <= max colour, and
    D/O within the contributors' depth range, on the 2,000-Gaussian scene."""
    w = synth.tiny()
    m, cam = w.gmap.as_dict(), w.cams[0]
    r = oracle.render(m, cam)
    p = oracle.project(m, cam)
    assert r["t_final"].min() >= 1e-4
    np.testing.assert_allclose(r["opac"], 1 - r["t_final"], atol=1e-13)
    assert r["rgb"].min() >= 0 and r["rgb"].max() <= p["rgb"][:, p["valid"] == 1].max() + 1e-12
    hit = r["opac"] > 0
    dd = r["depth"][hit] / r["opac"][hit]
    vd = p["depth"][p["valid"] == 1]
    assert dd.min() >= vd.min() - 1e-9 and dd.max() <= vd.max() + 1e-9
    assert (r["flags"] != 0).mean() < 0.01


def test_culling_is_lossless_and_lists_match_brute_force(oracle):
    """Footprint-enumerated render = every-Gaussian-at-every-pixel render, and
    tile lists from the footprint box = lists from testing every tile."""
    w = synth.tiny()
    m, cam = w.gmap.as_dict(), w.cams[0]
    r1 = oracle.render(m, cam)
    r2 = oracle.render(m, cam, brute=True)
    for k in ("rgb", "depth", "opac", "t_final", "n_contrib", "last_gid"):
        np.testing.assert_array_equal(r1[k], r2[k])
    t1 = oracle.tiles(m, cam)
    t2 = oracle.tiles(m, cam, brute=True)
    for a, b in zip(t1, t2):
        np.testing.assert_array_equal(a, b)
    # every pixel's last contributor is in the list of the pixel's tile
    tile, gid, margin = t1
    pairs = set(zip(tile.tolist(), gid.tolist()))
    tw = (cam["width"] + 15) // 16
    ys, xs = np.nonzero(r1["last_gid"] >= 0)
    for y, x in zip(ys, xs):
        assert ((y // 16) * tw + x // 16, int(r1["last_gid"][y, x])) in pairs
    # sorted by (tile, depth key, index)
    keys = oracle.depth_keys(m, cam)
    order = np.lexsort((gid, keys[gid], tile))
    np.testing.assert_array_equal(order, np.arange(len(tile)))


def test_permuting_gaussians_leaves_image_unchanged(oracle):
    w = synth.tiny(n=400)
    m, cam = w.gmap.as_dict(), w.cams[0]
    perm = np.random.default_rng(3).permutation(400)
    mp = synth.GaussianMap(**{k: v for k, v in m.items()}).subset(perm).as_dict()
    r1, r2 = oracle.render(m, cam), oracle.render(mp, cam)
    np.testing.assert_allclose(r1["rgb"], r2["rgb"], atol=1e-12)
    np.testing.assert_allclose(r1["depth"], r2["depth"], atol=1e-12)


def test_degree_zero_colour_is_view_independent(oracle):
    w = synth.tiny(n=200)
    m = w.gmap.as_dict()
    c1 = synth.camera(np.eye(3), [0, 0, 0], 100, 100, 64, 48, 128, 96)
    R, t = synth.pose_from_centre(synth.yaw_pitch_rotation(0.3, 0.1), (1.0, 0.5, -2.0))
    c2 = synth.camera(R, t, 100, 100, 64, 48, 128, 96)
    p1, p2 = oracle.project(m, c1), oracle.project(m, c2)
    both = (p1["valid"] == 1) & (p2["valid"] == 1)
    np.testing.assert_allclose(p1["rgb"][:, both], p2["rgb"][:, both], atol=1e-12)


# ---------------------------------------------------------------- loss
def test_loss_closed_forms(oracle):
    """L1 colour term = w mean |r| and depth term = w_d mean over D_s > 0 of
    |D/O - D_s| (Eq. depth_loss with means, O = 0 pixels contribute nothing)."""
    w = synth.tiny(n=500)
    m, cam = w.gmap.as_dict(), w.cams[0]
    r = oracle.render(m, cam)
    H, W = cam["height"], cam["width"]
    tgt = (r["rgb"] - 0.01)[None]
    b = oracle.backward(m, [cam], tgt_rgb=tgt, tgt_depth=np.zeros((1, H, W)), w_rgb=0.7, w_depth=0.3)
    assert b["loss"][0] == pytest.approx(0.7 * 0.01, rel=1e-9)
    mask = w.meta["depth_mask"][0]
    ds = np.where(mask, np.where(r["opac"] > 0, r["depth"] / np.maximum(r["opac"], 1e-300), 0) + 0.1, 0.0)
    b = oracle.backward(m, [cam], tgt_rgb=r["rgb"][None], tgt_depth=ds[None], w_rgb=0.7, w_depth=0.3)
    hit = (mask & (r["opac"] > 0)).sum()
    assert b["loss"][0] == pytest.approx(0.3 * 0.1 * hit / mask.sum(), rel=1e-9)


# ---------------------------------------------------------------- gradients
def _set(m, key, row, gi, delta):
    a = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    a = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in a.items()}
    if key == "logit_opacity":
        a[key][gi] += delta
    else:
        a[key].reshape(-1, a[key].shape[-1])[row, gi] += delta
    return a


def _get(g, key, row, gi):
    return g[key][gi] if key == "logit_opacity" else g[key].reshape(-1, g[key].shape[-1])[row, gi]


def test_gradients_match_central_differences(oracle):
    """Analytic gradients of a linear functional of (C, D, O) w.r.t. every
    parameter block equal FP64 central differences (step 1e-6), on samples
    whose contributor sets do not change between the two evaluations."""
    m, cam = small_scene()
    m = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(11)
    wr, wd, wo = rng.normal(size=(1, 3, H, W)), 0.05 * rng.normal(size=(1, H, W)), rng.normal(size=(1, H, W))

    def F(mm):
        r = oracle.render(mm, cam, margin_eps=0.0)
        return (wr[0] * r["rgb"]).sum() + (wd[0] * r["depth"]).sum() + (wo[0] * r["opac"]).sum(), r

    g = oracle.backward(m, [cam], ext_rgb=wr, ext_depth=wd, ext_opac=wo)
    touched = np.flatnonzero(np.abs(g["mean"]).sum(0) > 0)
    assert len(touched) > 50
    checked = 0
    for gi in rng.choice(touched, 10, replace=False):
        for key, rows in (("mean", 3), ("log_scale", 3), ("quat", 4), ("logit_opacity", 1), ("sh_dc", 3),
                          ("sh_rest", 45)):
            for row in rng.choice(rows, min(rows, 2), replace=False):
                h = 1e-6
                fp, rp = F(_set(m, key, row, gi, h))
                fm, rm = F(_set(m, key, row, gi, -h))
                if not np.array_equal(rp["n_contrib"], rm["n_contrib"]):
                    continue
                an = _get(g, key, row, gi)
                assert (fp - fm) / (2 * h) == pytest.approx(an, rel=2e-5, abs=2e-6), (key, row, gi)
                checked += 1
    assert checked >= 80


def _se3(xi):
    X = np.zeros((4, 4))
    rho, th = xi[:3], xi[3:]
    X[:3, :3] = [[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]]
    X[:3, 3] = rho
    return expm(X)


def _perturbed(cam, xi):
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = cam["R"], cam["t"]
    Tp = T @ _se3(xi)
    return dict(cam, R=Tp[:3, :3], t=Tp[:3, 3])


def test_pose_gradient_matches_se3_central_differences(oracle):
    """dL/dxi under T Exp(xi) (Eq. 3dgs_jacobi and the manifold derivative),
    Exp from scipy's matrix exponential of the twist.  Pixels whose
    contributor count differs between the +h and -h poses get zero weight."""
    m, cam = small_scene(seed=5)
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(2)
    wr, wd, wo = rng.normal(size=(1, 3, H, W)), 0.05 * rng.normal(size=(1, H, W)), rng.normal(size=(1, H, W))
    h = 1e-6
    renders = []
    keep = np.ones((H, W), bool)
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        rp = oracle.render(m, _perturbed(cam, xi), margin_eps=0.0)
        rm = oracle.render(m, _perturbed(cam, -xi), margin_eps=0.0)
        keep &= rp["n_contrib"] == rm["n_contrib"]
        renders.append((rp, rm))
    assert keep.mean() > 0.98
    wr, wd, wo = wr * keep, wd * keep, wo * keep
    g = oracle.backward(m, [cam], ext_rgb=wr, ext_depth=wd, ext_opac=wo)

    def F(r):
        return (wr[0] * r["rgb"]).sum() + (wd[0] * r["depth"]).sum() + (wo[0] * r["opac"]).sum()

    for k, (rp, rm) in enumerate(renders):
        assert (F(rp) - F(rm)) / (2 * h) == pytest.approx(g["pose"][0, k], rel=1e-5, abs=1e-4)


def test_pose_jacobian_rows_match_differences_and_reverse_mode(oracle):
    """Forward-mode rows dC_p/dxi equal SE(3) central differences of the
    rendered colour, and sum_p J_p^T g_p equals the reverse-mode pose gradient."""
    m, cam = small_scene(seed=9, n=300, width=48, height=40)
    H, W = cam["height"], cam["width"]
    pix = np.arange(H * W, dtype=np.int32)
    J, rgb = oracle.pose_jacobian(m, cam, pix)
    r0 = oracle.render(m, cam)
    np.testing.assert_allclose(rgb.T.reshape(3, H, W), r0["rgb"], atol=1e-13)
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = 1e-6
        rp, rm = oracle.render(m, _perturbed(cam, xi)), oracle.render(m, _perturbed(cam, -xi))
        same = (rp["n_contrib"] == rm["n_contrib"]).reshape(-1)
        fd = ((rp["rgb"] - rm["rgb"]) / 2e-6).reshape(3, -1).T
        np.testing.assert_allclose(J[same, :, k], fd[same], rtol=1e-5, atol=1e-5)
    gC = np.random.default_rng(4).normal(size=(1, 3, H, W))
    g = oracle.backward(m, [cam], ext_rgb=gC)
    want = np.einsum("pck,pc->k", J, gC[0].reshape(3, -1).T)
    np.testing.assert_allclose(g["pose"][0], want, rtol=1e-9, atol=1e-9)


def test_fused_loss_gradient_equals_external_adjoint(oracle):
    """The fused L1 + depth loss back-propagates the adjoints
    w sign(r)/(3HW), w_d sign(r)/(O |M_d|), -w_d sign(r) D/(O^2 |M_d|)."""
    w = synth.tiny(n=500)
    m, cam = w.gmap.as_dict(), w.cams[0]
    H, W = cam["height"], cam["width"]
    r = oracle.render(m, cam)
    mask = w.meta["depth_mask"][0]
    ds = np.where(mask, 6.0, 0.0)
    b1 = oracle.backward(m, [cam], tgt_rgb=w.tgt_rgb, tgt_depth=ds[None], w_rgb=1.0, w_depth=0.5)
    s = np.sign(r["rgb"] - w.tgt_rgb[0])
    hit = mask & (r["opac"] > 0)
    O = np.where(hit, r["opac"], 1.0)
    sd = np.where(hit, np.sign(r["depth"] / O - 6.0), 0.0)
    n = mask.sum()
    b2 = oracle.backward(m, [cam], ext_rgb=(s / (3 * H * W))[None], ext_depth=(0.5 * sd / (O * n))[None],
                         ext_opac=(-0.5 * sd * r["depth"] / (O * O * n))[None])
    for k in ("mean", "log_scale", "quat", "logit_opacity", "sh_dc"):
        np.testing.assert_allclose(b1[k], b2[k], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(b1["pose"], b2["pose"], rtol=1e-10, atol=1e-14)


def test_rigid_motion_of_world_and_camera_leaves_image_unchanged(oracle):
    """Moving every Gaussian by a rigid motion G (means G mu, rotations
    composed with scipy's Rotation) and the camera by T G^-1 renders the same
    image (degree-0 colours), for a rotated and translated camera."""
    from scipy.spatial.transform import Rotation
    w = synth.tiny(n=600)
    m = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in w.gmap.as_dict().items()}
    R0, t0 = synth.pose_from_centre(synth.yaw_pitch_rotation(0.2, -0.1, 0.05), (0.3, -0.2, -1.0))
    cam = synth.camera(R0, t0, 100, 100, 64, 48, 128, 96)
    rG = Rotation.from_rotvec([0.4, -0.7, 0.25])
    tG = np.array([1.5, -2.0, 0.7])
    m2 = dict(m)
    m2["mean"] = (rG.as_matrix() @ m["mean"]) + tG[:, None]
    q = m["quat"] / np.linalg.norm(m["quat"], axis=0)
    rq = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], 1))
    q2 = (rG * rq).as_quat()
    m2["quat"] = np.stack([q2[:, 3], q2[:, 0], q2[:, 1], q2[:, 2]])
    R0d, t0d = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
    cam2 = dict(cam, R=R0d @ rG.as_matrix().T, t=t0d - R0d @ rG.as_matrix().T @ tG)
    cam1 = dict(cam, R=R0d, t=t0d)
    r1, r2 = oracle.render(m, cam1, margin_eps=1e-6), oracle.render(m2, cam2, margin_eps=1e-6)
    ok = (r1["flags"] == 0) & (r2["flags"] == 0)
    assert ok.mean() > 0.99
    for k in ("depth", "opac"):
        np.testing.assert_allclose(r1[k][ok], r2[k][ok], atol=1e-9)
    np.testing.assert_allclose(r1["rgb"][:, ok], r2["rgb"][:, ok], atol=1e-9)


def test_anisotropic_image_closed_form_with_library_inverse(oracle):
    """alpha = o exp(-1/2 d^T inv(Sigma') d) with Sigma' from the rotated-
    anisotropic closed form and inv from numpy (pins the conic and its sign)."""
    f, W, H = 40.0, 64, 48
    cam = identity_camera(W, H, f)
    phi, sx, sy, d = 0.7, 0.4, 0.12, 4.0
    q = [math.cos(phi / 2), 0, 0, math.sin(phi / 2)]
    m = one_gaussian_map([[0, 0, d]], [[math.log(sx), math.log(sy), math.log(0.05)]], [logit(0.9)], [[0.3, 0.6, 0.9]],
                         [q])
    r = oracle.render(m, cam)
    R2 = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    S = (f / d) ** 2 * R2 @ np.diag([sx ** 2, sy ** 2]) @ R2.T + 0.3 * np.eye(2)
    Si = np.linalg.inv(S)
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    dx, dy = xx - W / 2, yy - H / 2
    a = 0.9 * np.exp(-0.5 * (Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy))
    a = np.where(a >= A_MIN, np.minimum(a, 0.99), 0)
    np.testing.assert_allclose(r["opac"], a, atol=1e-12)
    np.testing.assert_allclose(r["rgb"][2], 0.9 * a, atol=1e-12)
