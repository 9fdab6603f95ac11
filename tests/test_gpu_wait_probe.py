"""The library's device wait ends on its own (needs a GPU).

The only spin-wait in the library is the binning sort's look-back of a tile on
the tiles before it, bounded at 65536 polls.  gs_sort_wait_probe runs one pass
of that sort on a synthetic array; with its first tile never taken the wait of
the second tile runs out, the pass reports GS_ERR_TIMEOUT and returns, and
the GPU context stays usable.  No fault, trap or unbounded wait is involved:
every access of the pass stays in range either way.
"""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _run(skip_first_tile: bool):
    from paper_2507_04004_b300 import _native as N
    n = N.gs_sort_wait_probe_bytes()
    scratch = torch.zeros((n + 3) // 4, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    N.gs_sort_wait_probe(scratch, skip_first_tile, status, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return int(status.item()), time.time() - t0, scratch


def test_sort_pass_without_a_missing_tile_sorts_stably():
    from paper_2507_04004_b300 import _native as N
    code, _, s = _run(False)
    assert code == N.GS_OK
    items = 4096
    base = 64 + 6 * 256 + 6 * 2 * 256
    w = s.cpu().numpy().view(np.uint32)
    keys_in, key_out, val_out = w[base:base + items], w[base + 2 * items:base + 3 * items], w[base + 3 * items:base + 4 * items]
    order = np.argsort(keys_in & 255, kind="stable")
    assert np.array_equal(val_out, order)
    assert np.array_equal(key_out, keys_in[order])


def test_sort_wait_on_a_tile_nobody_takes_times_out():
    from paper_2507_04004_b300 import _native as N
    code, secs, _ = _run(True)
    assert code == N.GS_ERR_TIMEOUT
    assert secs < 10.0
    # the context is still usable: an ordinary pass right after succeeds
    code2, _, _ = _run(False)
    assert code2 == N.GS_OK
