"""The render server (adop_serve_*): continuous batching of requests of mixed
resolution over several resident clouds.  Each result must equal the same
render done alone through adop_render_forward (features within the FP32
tolerance); admission respects the memory budget; bounded waits, cancel and
malformed requests report their status without touching the GPU."""
import threading

import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, assert_close

pytestmark = pytest.mark.gpu

LEVELS = 4


def _clouds(torch, adop):
    out = []
    for n, seed in ((20000, 5), (60000, 6)):
        sc = scenes.tiny_spheres(n, 8, seed=seed)
        out.append((sc, adop.Points(torch.from_numpy(sc.xyz).cuda(),
                                    torch.from_numpy(sc.feat).cuda())))
    return out


def _random_cam(rng, k):
    w, h = [(64, 48), (160, 120), (320, 240), (97, 61), (256, 256)][k % 5]
    eye = np.array([np.cos(k), 0.3 * np.sin(3 * k), np.sin(k)]) * rng.uniform(2.2, 3.0) + 0.5
    R, t = scenes.look_at(eye, np.full(3, 0.5) + rng.normal(scale=0.05, size=3))
    cam = scenes.Camera(w, h, 0.9 * w, 0.9 * w, w / 2, h / 2, k1=0.02, R=R, t=t)
    cam.ev = float(rng.uniform(-1, 1))
    cam.wb = (float(rng.uniform(0.8, 1.2)), 1.0, float(rng.uniform(0.8, 1.2)))
    cam.vig_a = (-0.1, 0.0, 0.0)
    cam.epilogue = bool(k % 2)
    return cam


def _alone(adop, torch, pts, cam, flags):
    params = adop.Params(LEVELS, 0.01, 1e-3, None, flags)
    fr = adop.Frame.alloc(cam, 8, LEVELS, torch.float32, True, "cuda")
    ws = adop.alloc_workspace(pts, [cam], params, None, "cuda")
    adop.adop_render_forward(pts, [cam], params, [fr], ws)
    torch.cuda.synchronize()
    return np.concatenate([im.cpu().numpy().ravel() for im in fr.images])


def test_results_alone_equal_results_in_the_mix(adop):
    import torch
    clouds = _clouds(torch, adop)
    flags = adop.ADOP_FLAG_EPILOGUE
    # a budget that holds only a few requests at a time forces admission by memory
    srv = adop.Server(mem_budget_bytes=24 << 20, max_slots=6, streams=3, max_batch=4, levels=LEVELS,
                      flags=flags)
    ids = [srv.load_cloud(p) for _, p in clouds]
    rng = np.random.default_rng(1)
    reqs = []
    lock = threading.Lock()

    def client(tid):
        r = np.random.default_rng(100 + tid)
        for k in range(12):
            cam = _random_cam(r, k + 7 * tid)
            cid = ids[(k + tid) % 2]
            out = torch.empty(adop.output_numel(cam, 8, LEVELS), dtype=torch.float32, device="cuda")
            t = srv.submit(cid, cam, out)
            with lock:
                reqs.append((t, cid, cam, out))

    threads = [threading.Thread(target=client, args=(i,)) for i in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for t, _, _, _ in reqs:
        assert srv.wait(t, 60_000) == 0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["mem_in_use"] == 0
    assert st["mem_peak"] <= 24 << 20 and st["batches"] >= 1
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for t, cid, cam, out in reqs:
        ref = _alone(adop, torch, clouds[cid][1], cam, flags)
        assert_close(out.cpu().numpy(), ref, RTOL_FEAT_F32, f"request {t}")
        assert srv.latency_ms(t) > 0
    srv.close()


def test_batches_form_and_mix_clouds(adop):
    """Under a burst, requests are batched (more than one camera per launch,
    cameras of different clouds in one launch) and every result still equals
    the render done alone."""
    import torch
    clouds = _clouds(torch, adop)
    flags = adop.ADOP_FLAG_EPILOGUE
    # a batching window far longer than the burst's submission: batches fill up
    srv = adop.Server(mem_budget_bytes=512 << 20, max_slots=64, streams=2, max_batch=8, levels=LEVELS,
                      flags=flags, batch_window_us=50_000)
    ids = [srv.load_cloud(p) for _, p in clouds]
    rng = np.random.default_rng(3)
    cams = [_random_cam(rng, k) for k in range(32)]
    outs = [torch.empty(adop.output_numel(c, 8, LEVELS), dtype=torch.float32, device="cuda") for c in cams]
    reqs = [(srv.submit(ids[k % 2], c, o), k % 2, c, o) for k, (c, o) in enumerate(zip(cams, outs))]
    for t, _, _, _ in reqs:
        assert srv.wait(t, 60_000) == 0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["mem_in_use"] == 0
    assert st["mean_batch"] > 1.0, st
    assert st["mixed_batches"] >= 1, st
    for t, cid, cam, out in reqs:
        ref = _alone(adop, torch, clouds[cid][1], cam, flags)
        assert_close(out.cpu().numpy(), ref, RTOL_FEAT_F32, f"request {t}")
    srv.close()


def test_admission_timeout_cancel_and_bad_requests(adop):
    import torch
    clouds = _clouds(torch, adop)
    srv = adop.Server(mem_budget_bytes=400 << 20, max_slots=1, streams=1, max_batch=1, levels=LEVELS)
    cid = srv.load_cloud(clouds[1][1])
    big = scenes.Camera(1920, 1080, 1500.0, 1500.0, 960.0, 540.0, R=np.eye(3, dtype=np.float32),
                        t=np.array([-0.5, -0.5, 2.5], np.float32))
    outs = [torch.empty(adop.output_numel(big, 8, LEVELS), device="cuda") for _ in range(3)]
    tickets = [srv.submit(cid, big, o) for o in outs]
    # the last one is still queued behind two full-HD renders on one slot
    assert srv.wait(tickets[2], 0) == 5                 # ADOP_ERR_TIMEOUT
    assert srv.cancel(tickets[2]) in (0, 6)             # cancelled, or already admitted (BUSY)
    assert srv.wait(tickets[0], 60_000) == 0 and srv.wait(tickets[1], 60_000) == 0
    assert srv.poll(tickets[2]) in (0, 7)               # done or ADOP_ERR_CANCELLED
    # malformed requests are refused synchronously
    bad = scenes.Camera(0, 10, 1.0, 1.0, 0.0, 0.0)
    with pytest.raises(adop.AdopError, match="image size"):
        srv.submit(cid, bad, outs[0])
    nan = scenes.Camera(64, 48, float("nan"), 1.0, 0.0, 0.0)
    with pytest.raises(adop.AdopError, match="non-finite"):
        srv.submit(cid, nan, outs[0])
    with pytest.raises(adop.AdopError, match="unknown cloud"):
        srv.submit(7, big, outs[0])
    huge = scenes.Camera(16384, 16384, 1.0, 1.0, 0.0, 0.0)
    with pytest.raises(adop.AdopError, match="budget"):
        srv.submit(cid, huge, outs[0])
    srv.close()
    with pytest.raises(adop.AdopError):
        adop.Server(mem_budget_bytes=1024)
