"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): barrier,
max-over-ranks timing and the whole-job sum; replicas share no data."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    d = bench.Dist(use_cuda=False)
    d.barrier()
    t = d.max(10.0 + rank)
    s = d.sum(100.0 * (rank + 1))
    q.put((rank, t, s, d.rank, d.world))
    d.close()


def test_two_rank_max_and_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [300.0, 300.0]
    assert [(r[3], r[4]) for r in res] == [(0, 2), (1, 2)]


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, n = 1, 1, 10
    assert bench.run_reference(A()) == 0
