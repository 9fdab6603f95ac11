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


def test_reference_arm_prints_its_json_line():
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys; a small map and a few seconds of oracle
    time keep the test short."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "20000", "--steps", "2",
                        "--warmup", "1", "--reference-seconds", "3"], cwd=root, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Mpix/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
