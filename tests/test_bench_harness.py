"""The benchmark's multi-rank timing harness on CPU with 2 gloo ranks: each
rank times exactly K steps between barriers, and the reported time is the
maximum over ranks (replicas, no data exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist, r, w = bench.dist_setup("gloo")
    assert (r, w) == (rank, world)
    calls = []

    def step():
        calls.append(1)
        time.sleep(0.01 * (rank + 1))

    total, per = bench.timed_steps(step, 5, None, dist, "cpu")
    tmax = bench.max_over_ranks(dist, total, "cpu")
    out.put((rank, len(calls), total, tmax, len(per)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5, 5] and [r[4] for r in res] == [5, 5]
    slow = max(r[2] for r in res)
    assert all(abs(r[3] - slow) < 1e-9 for r in res)
    assert res[1][2] > res[0][2]


def test_algorithmic_bytes_model():
    import bench
    n, px, c = 1000, 500, 8
    assert bench.algorithmic_bytes("depth", n, px, c, 2, 2) == n * 12 + px * 16
    # the backward point pass reads and writes only the points in some Lambda
    assert bench.algorithmic_bytes("bwd_points", n, px, c, 2, 2, 400) == \
        400 * (4 + 4 + 12 + 16 + 32 + 12) + px * 48 + n * 4 + 600 * (32 + 12)
    assert bench.algorithmic_bytes("bwd_bin", n, px, c, 2, 2, 400) == n * 8 + 400 * 4
    with pytest.raises(KeyError):
        bench.algorithmic_bytes("nope", n, px, c, 2, 2)
