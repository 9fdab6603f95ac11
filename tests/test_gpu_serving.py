"""Continuous-batching server (needs a GPU): every request's result is the
same alone (plain one-launch-per-request path) and inside a mixed, batched,
overlapping stream; the sort-buffer budget bounds what is in flight."""
import numpy as np
import pytest
import torch

from paper_2507_04004_b300 import synth

pytestmark = pytest.mark.gpu


def _requests(rng, n, box_lo, box_hi):
    from paper_2507_04004_b300.serve import Request
    sizes = [(160, 96), (320, 176), (480, 272)]
    reqs = []
    img = synth.smooth_target(rng, 96, 128)
    pix = synth.top_gradient_pixels(img, 500)
    tgt = img.reshape(3, -1)[:, pix].T.copy()
    for i, (centre, Rc) in enumerate(synth.tracking_poses(rng, n, box_lo, box_hi)):
        R, t = synth.pose_from_centre(Rc, centre)
        if i % 3 == 2:
            cam = synth.camera(R, t, 100.0, 100.0, 64, 48, 128, 96)
            reqs.append(Request("jacobian", cam, pix=pix, target=tgt))
        else:
            W, H = sizes[i % len(sizes)]
            cam = synth.camera(R, t, 0.6 * W, 0.6 * W, W / 2, H / 2, W, H)
            reqs.append(Request("render", cam))
    return reqs


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_alone_equal_results_in_the_mix(use_graphs):
    from paper_2507_04004_b300.raster import GaussianMap
    from paper_2507_04004_b300.serve import PlainRenderer, Server
    rng = np.random.default_rng(1)
    lo, hi = (-6.0, -2.0, -6.0), (6.0, 2.0, 6.0)
    g = synth.random_map(rng, 30000, lo, hi, 3, log_scale_mean=-2.3)
    gm = GaussianMap.from_host(g, sh_bf16=True)
    reqs = _requests(rng, 24, lo, hi)
    budget = 64 << 20
    srv = Server(gm, mem_budget=budget, max_views=4, n_streams=3, use_graphs=use_graphs, pairs_per_pixel=6.0)
    srv.calibrate(reqs[:3])
    srv.warmup({r.key for r in reqs})
    srv.start()
    futs = [srv.submit(r) for r in reqs]  # all at once: batches form and overlap
    res = [f.result(timeout=120) for f in futs]
    srv.stop()
    assert srv.batches < len(reqs)
    assert srv.max_inflight_bytes <= max(budget, max(r.bytes for rs in srv.runners.values() for r in rs))
    plain = PlainRenderer(gm)
    checked = PlainRenderer(gm, checked=True)
    for r, got in zip(reqs, res):
        alone = plain.run(r)
        simple = checked.run(r)  # the plain loop with a status read-back between sort and blend
        for k in alone:
            assert np.array_equal(alone[k], simple[k])
        if r.kind == "render":
            assert np.array_equal(got["rgb"], alone["rgb"]) and np.array_equal(got["depth"], alone["depth"])
        else:
            assert np.array_equal(got["rgb"], alone["rgb"])
            scale = np.abs(alone["J"]).max()
            assert np.abs(got["J"] - alone["J"]).max() <= 1e-3 * scale
            np.testing.assert_allclose(got["residual"], alone["rgb"] - r.target, atol=1e-6)


def test_runners_built_while_serving_give_the_same_results():
    """Warm-up without multi-view runners, then a burst of one request kind:
    the runners for larger batches are created while batches are in flight
    (on the builder thread), and every result still equals the request
    rendered alone."""
    from paper_2507_04004_b300.raster import GaussianMap
    from paper_2507_04004_b300.serve import PlainRenderer, Request, Server
    rng = np.random.default_rng(2)
    lo, hi = (-6.0, -2.0, -6.0), (6.0, 2.0, 6.0)
    g = synth.random_map(rng, 30000, lo, hi, 3, log_scale_mean=-2.3)
    gm = GaussianMap.from_host(g, sh_bf16=True)
    reqs = []
    for centre, Rc in synth.tracking_poses(rng, 40, lo, hi):
        R, t = synth.pose_from_centre(Rc, centre)
        reqs.append(Request("render", synth.camera(R, t, 190.0, 190.0, 160, 88, 320, 176)))
    srv = Server(gm, mem_budget=1 << 30, max_views=4, n_streams=3, pairs_per_pixel=6.0)
    srv.calibrate(reqs[:2])
    srv.warmup({reqs[0].key}, copies=0)  # two single-view runners only
    srv.start(prime=reqs[:1])
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=120) for f in futs]
    srv.stop()
    assert srv.runners_added >= 1 and any(s > 1 for *_, s in srv.added_keys)
    plain = PlainRenderer(gm)
    for r, got in zip(reqs, res):
        alone = plain.run(r)
        assert np.array_equal(got["rgb"], alone["rgb"]) and np.array_equal(got["depth"], alone["depth"])
