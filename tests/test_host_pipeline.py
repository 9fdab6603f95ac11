"""Host side of the keyframe upload (no GPU): 8-bit targets survive the
byte round trip exactly, and the sparse depth packing reproduces the dense
depth maps, including a view without any LiDAR point."""
import numpy as np
import torch

from paper_2507_04004_b300 import synth
from paper_2507_04004_b300.pipeline import HostKeyframes, pack_sparse_depth


def test_8bit_round_trip_is_exact():
    rng = np.random.default_rng(5)
    img = synth.quantize_8bit(rng.random((2, 3, 17, 23)) * 1.2 - 0.1)
    b = synth.to_uint8(img)
    assert b.dtype == np.uint8 and b.min() == 0 and b.max() == 255
    np.testing.assert_array_equal(b.astype(np.float32) / np.float32(255.0), img)
    k = np.arange(256)
    np.testing.assert_array_equal(synth.to_uint8(synth.quantize_8bit(k / 255.0)), k)


def test_sparse_depth_packing_reproduces_the_maps():
    rng = np.random.default_rng(6)
    V, H, W = 3, 19, 31
    depth = np.where(rng.random((V, H, W)) < 0.05, rng.uniform(0.5, 80.0, (V, H, W)), 0.0).astype(np.float32)
    depth[1] = 0.0                                   # a view without depth
    depth[2, -1, -1] = 7.25                          # the last pixel
    idx, val, offs = pack_sparse_depth(depth)
    assert idx.dtype == np.int32 and val.dtype == np.float32 and offs.dtype == np.int32
    assert offs[0] == 0 and offs[-1] == idx.size == int((depth > 0).sum()) and offs[2] == offs[1]
    back = np.zeros((V, H * W), np.float32)
    for v in range(V):
        back[v, idx[offs[v]:offs[v + 1]]] = val[offs[v]:offs[v + 1]]
        assert np.all(np.diff(idx[offs[v]:offs[v + 1]]) > 0)
    np.testing.assert_array_equal(back.reshape(V, H, W), depth)
    kf = HostKeyframes.from_dense(np.zeros((V, 3, H, W), np.uint8), depth, torch.zeros(V, 16), pin=False)
    assert kf.nbytes() == V * 3 * H * W + 8 * idx.size + 4 * (V + 1) + 4 * 16 * V
