"""Sparse Adam through the C ABI (needs a GPU): exactly the Gaussians the
projection saw are updated, by the Adam recurrence, and their gradients are
cleared; the rest of the map and its moments stay as they were.  Which
Gaussians are seen is decided by the oracle's projection on a scene built so
that it is unambiguous (half the Gaussians well inside the frustum, half
behind the camera); the gradients are seeded random arrays."""
import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import synth
from tests.gpu_cases import host_map

pytestmark = pytest.mark.gpu

FIELDS = ("mean", "log_scale", "quat", "logit_opacity", "sh_dc", "sh_rest")


def test_sparse_adam_updates_the_seen_gaussians(oracle):
    from paper_2507_04004_b300.raster import GaussianMap, Rasterizer, SparseAdam, cameras_tensor
    rng = np.random.default_rng(30)
    n = 3000
    g = synth.random_map(rng, n, (-1, -1, 4), (1, 1, 8), 2, log_scale_mean=-2.5)
    behind = rng.random(n) < 0.5
    g.mean[2, behind] = -g.mean[2, behind]
    cam = synth.camera(np.eye(3), np.zeros(3), 100.0, 100.0, 64.0, 48.0, 128, 96)
    seen = oracle.project(host_map(g), cam)["valid"].astype(bool)
    assert seen.sum() > 1000 and np.array_equal(seen, ~behind)
    gm = GaussianMap.from_host(g)
    rast = Rasterizer(gm.n, 1, 128, 96)
    rast.project_and_sort(gm, cameras_tensor([cam]))
    lrs = dict(mean=0.01, log_scale=0.02, quat=0.03, logit_opacity=0.04, sh_dc=0.05, sh_rest=0.06)
    opt = SparseAdam(gm, lr_mean=lrs["mean"], lr_log_scale=lrs["log_scale"], lr_quat=lrs["quat"],
                     lr_logit_opacity=lrs["logit_opacity"], lr_sh_dc=lrs["sh_dc"], lr_sh_rest=lrs["sh_rest"],
                     eps=1e-8)
    p_ref = {k: getattr(gm, k).cpu().numpy().astype(np.float64) for k in FIELDS}
    m_ref = {k: np.zeros_like(v) for k, v in p_ref.items()}
    v_ref = {k: np.zeros_like(v) for k, v in p_ref.items()}
    grads = None
    for step in (1, 2):
        gr = {k: rng.normal(size=p_ref[k].shape).astype(np.float32) for k in FIELDS}
        from paper_2507_04004_b300.raster import Grads
        grads = Grads(*(torch.as_tensor(gr[k], device="cuda") for k in FIELDS), torch.zeros(1, 6, device="cuda"),
                      torch.zeros(1, device="cuda"))
        opt.step(gm, grads, rast)
        for k in FIELDS:
            gk = gr[k].astype(np.float64)
            sel = np.zeros(p_ref[k].shape, bool)
            sel[..., seen] = True
            m_new = 0.9 * m_ref[k] + 0.1 * gk
            v_new = 0.999 * v_ref[k] + 0.001 * gk * gk
            upd = lrs[k] * (m_new / (1 - 0.9 ** step)) / (np.sqrt(v_new / (1 - 0.999 ** step)) + 1e-8)
            p_ref[k] = np.where(sel, p_ref[k] - upd, p_ref[k])
            m_ref[k] = np.where(sel, m_new, m_ref[k])
            v_ref[k] = np.where(sel, v_new, v_ref[k])
            np.testing.assert_allclose(getattr(gm, k).cpu().numpy(), p_ref[k], rtol=1e-5, atol=1e-6, err_msg=k)
            np.testing.assert_allclose(getattr(opt.m, k).cpu().numpy(), m_ref[k], rtol=1e-5, atol=1e-7, err_msg=k)
            got_g = getattr(grads, k).cpu().numpy()
            assert not np.any(got_g[..., seen]), k                          # cleared where updated
            np.testing.assert_array_equal(got_g[..., ~seen], gr[k][..., ~seen])  # untouched elsewhere
    assert int(opt.step_count.item()) == 2
