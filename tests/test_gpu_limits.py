"""The ABI's limits, at the limit: 64 cameras in one call (ADOP_MAX_CAMERAS,
i.e. four launches of 16), and one 16384 x 16384 camera (the largest image)
with 8 pyramid layers (ADOP_MAX_LEVELS), against the oracle."""
import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, compare, gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu


def test_sixty_four_cameras_in_one_call(adop, orc):
    sc = scenes.tiny_spheres(20000, 4, seed=601)
    res = ((64, 48), (97, 61), (128, 96), (50, 33))
    cams = scenes.orbit_cameras(adop.ADOP_MAX_CAMERAS, seed=602, radius=2.5, resolutions=res, photometric=False)
    for cam in cams:
        R, t = scenes.look_at(-cam.R.T @ cam.t, np.full(3, 0.5))
        cam.R, cam.t = R, t
    G = [scenes.upstream_grad(c.w, c.h, 4, sc.c, 700 + k) for k, c in enumerate(cams)]
    g = gpu_run(adop, sc, cams, "f32", grads=G)
    r = oracle_run(orc, sc, cams, "f32", grads=G)
    compare(g, r)
    assert all(np.count_nonzero(c) > 0 for c in g["cnt"])


def test_largest_image_and_deepest_pyramid(adop, orc):
    import torch
    levels = adop.ADOP_MAX_LEVELS
    w = h = 16384
    sc = scenes.surfaces_scene(2_000_000, 1, seed=603, size_scale=scenes.SIZE_SCALE_SINGLE_VIEW)
    cam = scenes.single_view_camera(w, h, seed=604, f=0.6 * w)
    pts = adop.Points(torch.from_numpy(sc.xyz).cuda(), torch.from_numpy(sc.feat).cuda())
    params = adop.Params(levels, 0.01, 1e-3, None, 0)
    fr = adop.Frame.alloc(cam, 1, levels, torch.float32, True, "cuda")
    ws = adop.alloc_workspace(pts, [cam], params, None, "cuda")
    adop.adop_render_forward(pts, [cam], params, [fr], ws)
    torch.cuda.synchronize()
    keys = fr.key.cpu().numpy().view(np.uint64)
    cnt = fr.count.cpu().numpy().view(np.uint32)
    imgs = [im.cpu().numpy() for im in fr.images]
    del pts, fr, ws
    torch.cuda.empty_cache()
    r = orc.keys_counts(sc.xyz, cam, levels)
    assert np.array_equal(keys, r.keys), f"{np.count_nonzero(keys != r.keys)} keys differ"
    assert np.array_equal(cnt, r.cnt)
    # the image at sampled pixels of every layer, against the mean over Lambda
    rng = np.random.default_rng(605)
    a1 = np.float32(1.0) + np.float32(0.01)
    off = 0
    for l in range(levels):
        wl, hl = w >> l, h >> l
        hit = np.flatnonzero(r.cnt[off:off + wl * hl])
        assert hit.size > 0, l
        sample = np.sort(rng.choice(hit, min(300, hit.size), replace=False))
        pl = r.pix[:, l]
        sel = np.flatnonzero(np.isin(pl, sample))
        zmin = (r.keys[off + pl[sel]] >> np.uint64(32)).astype(np.uint32).view(np.float32)
        inl = sel[r.z[sel] <= zmin * a1]
        idx = np.searchsorted(sample, pl[inl])
        ref = np.zeros(sample.size)
        n = np.zeros(sample.size)
        np.add.at(ref, idx, sc.feat[inl, 0].astype(np.float64))
        np.add.at(n, idx, 1.0)
        assert np.array_equal(n, r.cnt[off + sample])
        got = imgs[l].reshape(-1)[sample]
        assert rel_err(got, ref / n) <= RTOL_FEAT_F32, l
        off += wl * hl
