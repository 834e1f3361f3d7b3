"""The environment map on the GPU (Sec. 3.1): empty pixels sample a spherical
map along their ray, the spatial gradient's empty-target case uses that value,
and adop_env_backward scatters dL/dE into the texels.  Everything against the
oracle on the same seeded inputs, with the tolerances derived in parity.py."""
import numpy as np
import pytest

import scenes
from parity import (RTOL_ENV_GRAD, RTOL_ENV_IMG, RTOL_FEAT_F32, assert_close, compare, epilogue_decidable_grads,
                    gpu_run, oracle_run)

pytestmark = pytest.mark.gpu


def _cams(model=0):
    cams = scenes.orbit_cameras(2, seed=81, radius=2.5, resolutions=((128, 96), (100, 75)))
    for cam in cams:
        R, t = scenes.look_at(-cam.R.T @ cam.t, np.full(3, 0.5))
        cam.R, cam.t = R, t
        if model == 1:
            w, h = cam.w, cam.h
            cam.model, cam.fx, cam.fy, cam.cx, cam.cy = 1, 0.45 * w, 0.45 * w, w / 2 + 0.3, h / 2 - 0.2
            # k2 >= 0 keeps the radial polynomial monotone over the whole image: every
            # pixel then has a ray (beyond the fold of the polynomial none does)
            cam.k1, cam.k2, cam.k3, cam.p1, cam.p2 = 0.03, 0.002, 0.0, 0.0, 0.0
    return cams


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_env_forward_backward(adop, orc, dtype):
    sc = scenes.tiny_spheres(6000, 4, seed=82)
    cams = _cams()
    env = scenes.env_map(4, 64, 128, seed=83)
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 84 + k) for k, c in enumerate(cams)]
    g = gpu_run(adop, sc, cams, dtype, grads=G, env=env)
    r = oracle_run(orc, sc, cams, dtype, grads=G, env=env)
    for k in range(len(cams)):
        empty = (r["cnt"][k] == 0).sum()
        assert 0.2 * r["cnt"][k].size < empty < 0.95 * r["cnt"][k].size
    errs = compare(g, r, dtype, env=True)
    assert np.abs(r["denv"]).max() > 0 and errs["denv"] <= RTOL_ENV_GRAD


def test_env_without_kept_state(adop, orc):
    # the backward re-renders the pixel state and samples the map itself
    sc = scenes.tiny_spheres(6000, 4, seed=101)
    cams = _cams()
    env = scenes.env_map(4, 64, 128, seed=102)
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 103 + k) for k, c in enumerate(cams)]
    g = gpu_run(adop, sc, cams, "f32", grads=G, env=env, keep_state=False)
    r = oracle_run(orc, sc, cams, "f32", grads=G, env=env)
    compare(g, r, check_state=False, env=True)


def test_env_fisheye(adop, orc):
    sc = scenes.tiny_spheres(6000, 4, seed=85)
    cams = _cams(model=1)
    env = scenes.env_map(4, 64, 128, seed=86)
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 87 + k) for k, c in enumerate(cams)]
    g = gpu_run(adop, sc, cams, "f32", grads=G, env=env)
    r = oracle_run(orc, sc, cams, "f32", grads=G, env=env)
    compare(g, r, env=True)


def test_env_with_photometric_epilogue(adop, orc):
    # the environment map's gradient at layer 0 is chained through the epilogue
    sc = scenes.tiny_spheres(6000, 4, seed=88)
    sc.feat = np.abs(sc.feat) * 0.6
    cams = _cams()
    env = scenes.env_map(4, 64, 128, seed=89)
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 90 + k) for k, c in enumerate(cams)]
    G = epilogue_decidable_grads(orc, sc, cams, G, env=env)
    g = gpu_run(adop, sc, cams, "f32", grads=G, env=env, flags=adop.ADOP_FLAG_EPILOGUE)
    r = oracle_run(orc, sc, cams, "f32", grads=G, env=env, epilogue=True)
    compare(g, r, env=True)


def test_env_without_points(adop, orc):
    sc = scenes.tiny_spheres(0, 3, seed=91)
    cams = _cams()[:1]
    env = scenes.env_map(3, 32, 64, seed=92)
    G = [scenes.upstream_grad(c.w, c.h, 4, 3, 93) for c in cams]
    g = gpu_run(adop, sc, cams, "f32", grads=G, env=env)
    r = oracle_run(orc, sc, cams, "f32", grads=G, env=env)
    assert not r["cnt"][0].any()
    assert_close(g["img"][0], r["img"][0], RTOL_ENV_IMG, "image")
    assert_close(g["denv"], r["denv"], RTOL_ENV_GRAD, "dL/dE")


def test_constant_env_equals_background(adop):
    sc = scenes.tiny_spheres(6000, 3, seed=94)
    cams = _cams()
    bg = np.array([0.2, -0.4, 0.9], np.float32)
    env = np.broadcast_to(bg[:, None, None], (3, 16, 32)).copy()
    G = [scenes.upstream_grad(c.w, c.h, 4, 3, 95 + k) for k, c in enumerate(cams)]
    a = gpu_run(adop, sc, cams, "f32", grads=G, background=bg)
    b = gpu_run(adop, sc, cams, "f32", grads=G, env=env)
    for k in range(len(cams)):
        assert np.array_equal(a["cnt"][k], b["cnt"][k])
        assert np.allclose(a["img"][k], b["img"][k], rtol=0, atol=1e-6)
    assert np.allclose(a["dxyz"], b["dxyz"], rtol=1e-5, atol=1e-5 * np.abs(a["dxyz"]).max())


def test_env_in_the_server(adop):
    import torch
    sc = scenes.tiny_spheres(6000, 8, seed=96)
    cams = _cams()
    env = torch.from_numpy(np.ascontiguousarray(np.moveaxis(scenes.env_map(8, 64, 128, seed=97), 0, -1))).cuda()
    pts = adop.Points(torch.from_numpy(sc.xyz).cuda(), torch.from_numpy(sc.feat).cuda())
    params = adop.Params(4, 0.01, 1e-3, None, 0, 1.5, env)
    srv = adop.Server(mem_budget_bytes=64 << 20, max_slots=4, streams=2, max_batch=2, levels=4, env=env)
    try:
        cid = srv.load_cloud(pts)
        for cam in cams:
            fr = adop.Frame.alloc(cam, 8, 4, torch.float32, True, "cuda")
            ws = adop.alloc_workspace(pts, [cam], params, None, "cuda")
            adop.adop_render_forward(pts, [cam], params, [fr], ws)
            out = torch.empty(adop.output_numel(cam, 8, 4), device="cuda")
            t = srv.submit(cid, cam, out)
            assert srv.wait(t) == 0
            torch.cuda.synchronize()
            alone = np.concatenate([im.cpu().numpy().ravel() for im in fr.images])
            # the same render; only the order of the FP32 feature sums may differ
            assert_close(out.cpu().numpy(), alone, RTOL_FEAT_F32, "server vs alone")
    finally:
        srv.close()


def test_env_autograd(adop, orc):
    import torch
    from paper_2110_06635_gb300.autograd import rasterize
    sc = scenes.tiny_spheres(6000, 4, seed=98)
    cams = _cams()
    env_np = scenes.env_map(4, 64, 128, seed=99)
    env = torch.from_numpy(np.ascontiguousarray(np.moveaxis(env_np, 0, -1))).cuda().requires_grad_(True)
    xyz = torch.from_numpy(sc.xyz).cuda()
    feat = torch.from_numpy(sc.feat).cuda()
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 100 + k) for k, c in enumerate(cams)]
    imgs = rasterize(xyz, feat, cams, env=env)
    loss = sum((im * torch.from_numpy(np.ascontiguousarray(G[k][l], np.float32)).cuda()).sum()
               for k in range(len(cams)) for l, im in enumerate(imgs[k]))
    loss.backward()
    r = oracle_run(orc, sc, cams, "f32", grads=G, env=env_np, backward=True)
    assert_close(np.moveaxis(env.grad.cpu().numpy(), -1, 0), r["denv"], RTOL_ENV_GRAD, "dL/dE through autograd")
