"""Camera tracking with the map fixed (needs a GPU): the pose update
T0 Exp(xi) against the matrix exponential, the Adam step against its
definition, the gradient of the tracking loss (1/2 L1 + 1/2 D-SSIM) at a
perturbed pose against the FP64 oracle, and the 30-iteration tracker on the
32-frame tracking workload lowering the loss and the rotation error."""
import numpy as np
import pytest
import torch
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from oracle import ssim as S
from paper_2507_04004_b300 import synth
from tests.gpu_cases import GRAD_TOL, host_map, rel_err

pytestmark = pytest.mark.gpu


def _twist(xi):
    X = np.zeros((4, 4))
    r, w = xi[:3], xi[3:]
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = r
    return X


def test_pose_apply_matches_matrix_exponential():
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import cameras_tensor
    rng = np.random.default_rng(20)
    V = 9
    cams = []
    for v in range(V):
        R = Rotation.random(random_state=v).as_matrix()
        cams.append(synth.camera(R, rng.normal(size=3), 500.0, 510.0, 320.0, 256.0, 640, 512))
    xi = rng.normal(0, 0.05, (V, 6))
    xi[0] = 0.0
    xi[1, 3:] = [1e-6, -2e-6, 5e-7]   # the small-angle series
    xi[2, 3:] = [0.9, -1.2, 0.4]      # a large rotation
    c0 = cameras_tensor(cams)
    out = torch.empty_like(c0)
    N.gs_pose_apply(c0, torch.as_tensor(xi, dtype=torch.float32, device="cuda"), V, out,
                    torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    for v in range(V):
        T = np.eye(4)
        T[:3, :3] = np.asarray(cams[v]["R"], np.float64).reshape(3, 3)
        T[:3, 3] = cams[v]["t"]
        Tw = T @ expm(_twist(xi[v].astype(np.float32).astype(np.float64)))
        np.testing.assert_allclose(got[v, :9].reshape(3, 3), Tw[:3, :3], atol=2e-6)
        np.testing.assert_allclose(got[v, 9:12], Tw[:3, 3], atol=2e-6 * max(1.0, np.abs(Tw[:3, 3]).max()))
        np.testing.assert_array_equal(got[v, 12:], c0.cpu().numpy()[v, 12:])


def _se3(R, t):
    T = np.eye(4)
    T[:3, :3] = np.asarray(R, np.float64).reshape(3, 3)
    T[:3, 3] = np.asarray(t, np.float64).reshape(3)
    return T


def test_pose_residual_matches_matrix_logarithm():
    """gs_pose_residual against scipy's matrix logarithm of A^-1 B (A, B the
    world-to-camera poses, i.e. Log(T(t) T~^-1) with camera-to-world T), at
    relative rotations of 0, 1e-6, 0.3, pi/2, 2.5 and 3.1 rad; Exp(Log(.))
    through gs_pose_apply gives B back, and B = A Exp(xi) gives xi back."""
    from scipy.linalg import logm
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import cameras_tensor
    rng = np.random.default_rng(23)
    angles = [0.0, 1e-6, 0.3, np.pi / 2, 2.5, 3.1, 1e-3, 1.0]
    A, B = [], []
    for k, ang in enumerate(angles):
        Ra = Rotation.random(random_state=100 + k).as_matrix()
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        Rrel = Rotation.from_rotvec(ang * axis).as_matrix()
        ta = rng.normal(0, 5.0, 3)
        trel = rng.normal(0, 0.5, 3)
        A.append(synth.camera(Ra, ta, 500.0, 500.0, 320.0, 256.0, 640, 512))
        Tb = _se3(Ra, ta) @ _se3(Rrel, trel)
        B.append(synth.camera(Tb[:3, :3], Tb[:3, 3], 500.0, 500.0, 320.0, 256.0, 640, 512))
    V = len(angles)
    ca, cb = cameras_tensor(A), cameras_tensor(B)
    r = torch.empty(V, 6, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    N.gs_pose_residual(ca, cb, V, r, st)
    got = r.cpu().numpy().astype(np.float64)
    for v in range(V):
        Ta = _se3(A[v]["R"], A[v]["t"])  # the float32 values, in float64
        Tb = _se3(B[v]["R"], B[v]["t"])
        X = np.real(logm(np.linalg.inv(Ta) @ Tb))
        want = np.array([X[0, 3], X[1, 3], X[2, 3], X[2, 1], X[0, 2], X[1, 0]])
        scale = max(1.0, np.abs(want[:3]).max())
        np.testing.assert_allclose(got[v, 3:], want[3:], atol=2e-5, err_msg=f"theta, angle {angles[v]}")
        np.testing.assert_allclose(got[v, :3], want[:3], atol=2e-5 * scale, err_msg=f"rho, angle {angles[v]}")
        assert abs(np.linalg.norm(got[v, 3:]) - angles[v]) < 2e-5
    # Exp(Log(A^-1 B)) = A^-1 B: A Exp(r) reproduces B
    back = torch.empty_like(ca)
    N.gs_pose_apply(ca, r, V, back, st)
    np.testing.assert_allclose(back.cpu().numpy()[:, :12], cb.cpu().numpy()[:, :12], atol=5e-5)
    # B = A Exp(xi): the residual is xi (rotation angles below pi)
    xi = rng.normal(0, 0.3, (V, 6)).astype(np.float32)
    xi[0] = 0.0
    xi[1, 3:] = [2e-7, -1e-7, 3e-7]
    xi[2, 3:] = [1.2, -2.0, 1.5]  # |theta| = 2.77 rad
    xt = torch.as_tensor(xi, device="cuda")
    cx = torch.empty_like(ca)
    N.gs_pose_apply(ca, xt, V, cx, st)
    N.gs_pose_residual(ca, cx, V, r, st)
    np.testing.assert_allclose(r.cpu().numpy(), xi, atol=3e-5)


def test_adam_step_matches_definition():
    from paper_2507_04004_b300 import _native as N
    rng = np.random.default_rng(21)
    V = 200  # more than one thread per component of the single block
    lr = [1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3]
    cfg = N.gs_adam_config((N.C.c_float * 6)(*lr), 0.9, 0.999, 1e-8)
    t = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda")
    xi, m, s = t(rng.normal(size=(V, 6))), t(np.zeros((V, 6))), t(np.zeros((V, 6)))
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    x_ref = xi.cpu().numpy().astype(np.float64)
    m_ref = np.zeros((V, 6))
    s_ref = np.zeros((V, 6))
    for k in range(1, 4):
        g = rng.normal(size=(V, 6)) * 10 ** rng.uniform(-3, 1, (V, 6))
        gd = t(g)
        N.gs_adam_pose(xi, gd, m, s, step, V, cfg, torch.cuda.current_stream().cuda_stream)
        g = g.astype(np.float32).astype(np.float64)
        m_ref = 0.9 * m_ref + 0.1 * g
        s_ref = 0.999 * s_ref + 0.001 * g * g
        x_ref -= np.array(lr) * (m_ref / (1 - 0.9 ** k)) / (np.sqrt(s_ref / (1 - 0.999 ** k)) + 1e-8)
        assert np.abs(gd.cpu().numpy()).max() == 0.0  # cleared for the next backward pass
        assert int(step.item()) == k
    np.testing.assert_allclose(xi.cpu().numpy(), x_ref, rtol=1e-5, atol=1e-6)
    # the iterate of lowest loss is kept per view: losses 0.5, 0.2, 0.3 keep the iterate before the second step
    best_loss = t(np.full(V, np.inf))
    best_xi = t(np.zeros((V, 6)))
    kept = None
    for k, lval in enumerate([0.5, 0.2, 0.3]):
        before = xi.clone()
        N.gs_adam_pose(xi, t(rng.normal(size=(V, 6))), m, s, step, V, cfg, torch.cuda.current_stream().cuda_stream,
                       loss=t(np.full(V, lval)), best_loss=best_loss, best_xi=best_xi)
        if k == 1:
            kept = before.cpu().numpy()
    np.testing.assert_array_equal(best_xi.cpu().numpy(), kept)
    np.testing.assert_allclose(best_loss.cpu().numpy(), 0.2, rtol=1e-7)


def test_tracking_loss_gradient_vs_oracle(oracle):
    """One tracking iteration's chain on the tiny scene: T0 Exp(xi), render,
    1/2 D-SSIM adjoint, fused 1/2 L1, pose-only backward."""
    from paper_2507_04004_b300 import _native as N
    from paper_2507_04004_b300.raster import DSSIM, GaussianMap, Rasterizer, cameras_tensor
    w = synth.tiny()
    m = host_map(w.gmap)
    cam0 = w.cams[0]
    tgt = oracle.render(m, cam0)["rgb"].astype(np.float32)  # target: the oracle's image at the true pose
    xi = np.array([0.01, -0.02, 0.015, 0.004, -0.006, 0.003])
    gm = GaussianMap.from_host(w.gmap)
    rast = Rasterizer(gm.n, 1, 128, 96)
    c0 = cameras_tensor([cam0])
    cams = torch.empty_like(c0)
    st = torch.cuda.current_stream().cuda_stream
    N.gs_pose_apply(c0, torch.as_tensor(xi[None], dtype=torch.float32, device="cuda"), 1, cams, st)
    out = rast.render(gm, cams)
    td = torch.as_tensor(tgt[None], device="cuda")
    g = rast.new_grads(gm)
    dl = torch.zeros_like(out.rgb)
    DSSIM(1, 96, 128)(out.rgb, td, 0.5, loss=g.loss, dl_dimg=dl)
    rast.backward(gm, cams, out, tgt_rgb=td, w_rgb=0.5, w_depth=0.0, dl_drgb=dl, grads=g, params=False)
    # oracle: the same pose in FP64, image, loss adjoint, pose gradient
    R, t = synth.se3_right_perturb(np.asarray(cam0["R"], np.float64).reshape(3, 3), np.asarray(cam0["t"]), xi)
    camx = dict(cam0, R=R, t=t)
    r = oracle.render(m, camx)
    img = r["rgb"]
    n = img.size
    adj = 0.5 * np.sign(img - tgt) / n + 0.5 * S.dssim_grad(img, tgt)
    o = oracle.backward(m, [camx], ext_rgb=adj[None])
    loss_o = 0.5 * np.abs(img - tgt).mean() + 0.5 * S.dssim(img, tgt)
    assert g.loss.item() == pytest.approx(loss_o, rel=1e-4)
    assert rel_err(g.pose.cpu().numpy()[0], o["pose"][0]) <= GRAD_TOL


def test_tracker_reduces_pose_error_on_the_tracking_workload():
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, cameras_tensor
    from paper_2507_04004_b300.track import PoseTracker
    w = synth.tracking()
    gm = GaussianMap.from_host(w.gmap)
    V, H, W = 32, 512, 640
    gt = cameras_tensor(w.meta["gt_cams"])
    r = Rasterizer(gm.n, V, W, H)
    targets = r.render(gm, gt).rgb.clone()  # images at the true poses
    del r
    tr = PoseTracker(gm, V, W, H, iters=30)
    xi, loss = tr.track(cameras_tensor(w.cams), targets)
    xi = xi.cpu().numpy().astype(np.float64)
    loss = loss.cpu().numpy()
    true = -w.meta["xi"]  # query = GT Exp(xi_q), so GT = query Exp(-xi_q)
    e0_rot = np.linalg.norm(true[:, 3:], axis=1)
    e1_rot = np.linalg.norm(xi[:, 3:] - true[:, 3:], axis=1)
    e0_tr = np.linalg.norm(true[:, :3], axis=1)
    e1_tr = np.linalg.norm(xi[:, :3] - true[:, :3], axis=1)
    assert np.all(np.isfinite(xi)) and np.all(np.isfinite(loss))
    # the kept iterate is the one of lowest loss; in this scene (a uniform cloud of Gaussians around the
    # camera) the loss falls steeply while the pose error falls mostly in rotation
    assert np.mean(loss.min(0) < 0.7 * loss[0]) >= 0.75
    assert np.mean(e1_rot < e0_rot) >= 0.8
    assert np.median(e1_rot) < 0.8 * np.median(e0_rot)
    assert np.median(e1_tr) <= 1.1 * np.median(e0_tr)
    # the factor-graph residual Log(T(t) T~^-1) against the poses tracking started from is the kept xi;
    # against the true poses it is the remaining pose error, smaller in rotation than at the start
    r = tr.residual().cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(r, xi, atol=3e-5)
    r_gt = tr.residual(gt).cpu().numpy().astype(np.float64)
    assert np.median(np.linalg.norm(r_gt[:, 3:], axis=1)) < 0.8 * np.median(e0_rot)
    # a second batch replays the captured graph and gives the same result
    xi2, _ = tr.track(cameras_tensor(w.cams), targets)
    np.testing.assert_allclose(xi2.cpu().numpy(), xi, rtol=0, atol=1e-5)
