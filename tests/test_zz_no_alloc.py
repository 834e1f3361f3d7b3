"""The allocation-free backward entry point (adop_render_backward_noalloc).

Some callers cannot call cudaMalloc: a renderer embedded in a host
application that owns all device memory through its own pool and forbids
allocations on its frame loop (an allocation can synchronise the device and
stall a frame), or a process whose device-memory budget is fixed up front.
For them the library keeps its backward scratch in one static device array.
The tests call that entry point through the C ABI twice in a row and check
each result against the workspace-taking adop_render_backward on the same
inputs, and against the FP64 CPU oracle directly, within the tolerances of
the parity tests; and they check the defining property -- one call after a
warm-up leaves the device's free memory unchanged.  They live in a file of
their own that is collected last, and need no state from other tests.
"""
import numpy as np
import pytest

import scenes
from parity import RTOL_GRAD, assert_close, assert_reduced, oracle_run

pytestmark = pytest.mark.gpu


def _setup(adop, sc, cams, levels=4):
    import torch
    dev = "cuda"
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(levels, 0.01, 1e-3, None, 0)
    frames = [adop.Frame.alloc(c, sc.c, levels, torch.float32, True, dev) for c in cams]
    ws = adop.alloc_workspace(pts, cams, params, None, dev)
    adop.adop_render_forward(pts, cams, params, frames, ws)
    G = [[torch.from_numpy(g).to(dev) for g in scenes.upstream_grad(c.w, c.h, levels, sc.c, 90 + k)]
         for k, c in enumerate(cams)]
    return pts, params, frames, ws, G


def _grads(adop, sc, cams, pts, params, frames, G, ws=None):
    import torch
    dev = "cuda"
    out = [torch.zeros((sc.n, sc.c), device=dev), torch.zeros((sc.n, 3), device=dev),
           torch.zeros((len(cams), 6), device=dev), torch.zeros((len(cams), 6), device=dev)]
    if ws is None:
        adop.adop_render_backward_noalloc(pts, cams, params, frames, G, *out)
    else:
        adop.adop_render_backward(pts, cams, params, frames, G, *out, ws)
    torch.cuda.synchronize()
    return [t.cpu().numpy().astype(np.float64) for t in out]


def _check(ref, got):
    assert_close(got[0], ref[0], RTOL_GRAD, "dL/dtau")
    assert_close(got[1], ref[1], RTOL_GRAD, "dL/dx")
    scale_p = np.abs(ref[2]).max() + 1e-30
    scale_k = np.abs(ref[3]).max() + 1e-30
    assert_reduced(got[2], ref[2], np.full_like(ref[2], scale_p), what="dL/dxi")
    assert_reduced(got[3], ref[3], np.full_like(ref[3], scale_k), what="dL/dK")


@pytest.mark.parametrize("multi", [False, True])
def test_noalloc_backward_matches_workspace_backward(adop, multi):
    sc = scenes.tiny_spheres(20000, 4, seed=1001)
    cams = [scenes.tiny_camera()]
    if multi:
        R, t = scenes.look_at(np.array([2.0, 0.5, -1.0]), np.full(3, 0.5))
        cams.append(scenes.Camera(200, 150, 180.0, 180.0, 100.0, 75.0, k1=0.02, R=R, t=t))
    pts, params, frames, ws, G = _setup(adop, sc, cams)
    ref = _grads(adop, sc, cams, pts, params, frames, G, ws)
    assert np.abs(ref[1]).max() > 0 and np.abs(ref[2]).max() > 0
    for _ in range(2):  # two calls in a row share (and overwrite) the static scratch
        _check(ref, _grads(adop, sc, cams, pts, params, frames, G))


def test_noalloc_rejects_what_does_not_fit(adop):
    import torch
    sc = scenes.tiny_spheres(1000, 8, seed=3)
    big = scenes.Camera(1920, 1080, 1500.0, 1500.0, 960.0, 540.0, R=np.eye(3, dtype=np.float32),
                        t=np.array([0, 0, 2], np.float32))
    pts, params, frames, ws, G = _setup(adop, sc, [big])
    with pytest.raises(adop.AdopError, match="static array"):
        adop.adop_render_backward_noalloc(pts, [big], params, frames, G, torch.zeros((sc.n, 8), device="cuda"))
    stateless = [adop.Frame.alloc(big, 8, 4, torch.float32, False, "cuda")]
    with pytest.raises(adop.AdopError, match="kept key/count/acc"):
        adop.adop_render_backward_noalloc(pts, [big], params, stateless, G)


def test_noalloc_backward_matches_the_oracle(adop, orc):
    """Against the FP64 oracle itself: per-point gradients within 1e-4 of
    max(|ref|, rms), pose and intrinsics within 1e-4 of the summed absolute
    (point, layer) terms."""
    sc = scenes.tiny_spheres(20000, 4, seed=1001)
    cams = [scenes.tiny_camera()]
    pts, params, frames, ws, G = _setup(adop, sc, cams)
    Gh = [[g.cpu().numpy() for g in row] for row in G]
    r = oracle_run(orc, sc, cams, "f32", grads=Gh)
    for _ in range(2):
        got = _grads(adop, sc, cams, pts, params, frames, G)
        assert_close(got[0], r["dfeat"], RTOL_GRAD, "dL/dtau vs oracle")
        assert_close(got[1], r["dxyz"], RTOL_GRAD, "dL/dx vs oracle")
        assert_reduced(got[2][0], r["dpose"][0], r["dpose_abs"][0], what="dL/dxi vs oracle")
        assert_reduced(got[3][0], r["dintr"][0], r["dintr_abs"][0], what="dL/dK vs oracle")


def test_noalloc_call_allocates_no_device_memory(adop):
    """After one warm-up call (which may load the library's device code and
    place the static array), a further call leaves cudaMemGetInfo's free
    bytes unchanged."""
    import torch
    sc = scenes.tiny_spheres(20000, 4, seed=1001)
    cams = [scenes.tiny_camera()]
    pts, params, frames, ws, G = _setup(adop, sc, cams)
    out = [torch.zeros((sc.n, sc.c), device="cuda"), torch.zeros((sc.n, 3), device="cuda"),
           torch.zeros((1, 6), device="cuda"), torch.zeros((1, 6), device="cuda")]
    adop.adop_render_backward_noalloc(pts, cams, params, frames, G, *out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    adop.adop_render_backward_noalloc(pts, cams, params, frames, G, *out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
