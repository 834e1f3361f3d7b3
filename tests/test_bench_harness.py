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
    """The measurement plan's per-unit bytes: per point (forward 24 + c s,
    backward 24 + c s + 4 c, + 12 with a re-run depth pass) and per pyramid
    pixel; the per-kernel split adds up to the step."""
    import bench
    n, px, c = 1000, 500, 8
    # the plan's totals for C = 8: BF16 112 B and FP32 144 B per point
    assert sum(bench.s8d_point_bytes(8, 2)) == 112 and sum(bench.s8d_point_bytes(8, 4)) == 144
    assert bench.s8d_point_bytes(8, 2, recompute=True)[1] == 72 + 12
    assert bench.s8d_pixel_bytes(8, 2) == (8 + 4 + 32 + 4 + 32 + 16, 32)
    step = bench.s8d_step_bytes(n, px, c, 2, 2)
    assert step == n * 112 + px * (96 + 32)
    kernels = ("clear", "depth", "accumulate", "normalize", "bwd_prepass", "bwd_bin", "bwd_points", "bwd_reduce")
    assert sum(bench.s8d_kernel_bytes(k, n, px, c, 2, 2) for k in kernels) == step
    assert bench.s8d_kernel_bytes("bwd_prepass", n, px, c, 2, 2) == 0
    # the implementation's own traffic: the backward point pass reads and
    # writes only the points in some Lambda, plus its pixel records
    assert bench.implementation_bytes("depth", n, px, c, 2, 2) == n * 13 + px * 16
    assert bench.implementation_bytes("bwd_points", n, px, c, 2, 2, 400) == \
        400 * (4 + 4 + 12 + 16 + 32 + 12) + px * 48 + n * 4 + 600 * (32 + 12)
    assert bench.implementation_bytes("bwd_bin", n, px, c, 2, 2, 400) == n * 8 + 400 * 4
    # the binning's block table: 8 blocks per SM (at most 1536 rows in all) x 32x32 tiles, written and read once
    assert bench.bin_table_bytes(1920, 1080, 152) == 1216 * 60 * 34 * 4
    assert bench.bin_table_bytes(1920, 1080, 152, ncam=16) == 76 * 60 * 34 * 4
    assert bench.bin_table_bytes(1920, 1080, 400, ncam=2) == 768 * 60 * 34 * 4
    assert bench.implementation_bytes("bwd_bin", n, px, c, 2, 2, 400, 1000) == n * 8 + 400 * 4 + 2000


def test_clock_summary_merges_nvidia_smi_and_nvml():
    """The clock record of a timed region: nvidia-smi lines and NVML samples
    (reason bits decoded) merge into one median, maximum and reason set."""
    import bench
    cs = bench.ClockSampler("GPU-test")
    cs.lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active"]
    cs.nvml_samples = [(2070, 2070, 0), (2055, 2070, bench.Nvml.SW_POWER_CAP), (2070, 2070, 0)]
    s = cs.summary()
    assert s["samples"] == 4 and s["samples_nvidia_smi"] == 1 and s["samples_nvml"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    cs.nvml_samples = [(1500, 2070, bench.Nvml.HW_SLOWDOWN | bench.Nvml.HW_THERMAL | bench.Nvml.SW_THERMAL)]
    cs.lines = []
    s = cs.summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_tools():
    """Where neither nvidia-smi nor NVML exists (this CPU container), the
    sampler records why and reports the region as unsampled."""
    import bench
    with bench.ClockSampler("GPU-none", poll_s=0.001) as cs:
        pass
    s = cs.summary()
    if s["samples"] == 0:
        assert s["reasons"] == ["unsampled"] and s["error"]
