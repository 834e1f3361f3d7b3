"""The oracle's thread count and point sample are aids for timing and for
clouds too large to visit in full; neither may change what it computes.

* Forward: keys, counts, images, pixels and depths are identical (bit for
  bit) for any thread count: each thread owns a range of pixels and takes
  the pairs landing there in the single-thread order.
* Backward: per-point outputs are identical for any thread count; the pose
  and intrinsics sums, added per thread and then over threads, agree with
  one thread's to FP64 rounding of the summed absolute terms.
* Sample: a sampled backward's rows equal the full backward's rows of the
  same points bit for bit, its other rows are zero, and the reduced sums of a
  partition of the points add up to the full sums.
"""
import numpy as np
import pytest

import scenes


def _scene():
    sc, cams = scenes.config(1)
    return sc, cams[0]


def _mid_scene():
    # a smaller cut of the single-view workload: many points per pixel, an
    # odd-sized image so that pixel ranges split layers unevenly
    sc = scenes.surfaces_scene(60_000, 8, seed=12, size_scale=scenes.SIZE_SCALE_SINGLE_VIEW)
    R, t = scenes.look_at(np.array([0.0, 2.0, -12.0]), np.zeros(3))
    cam = scenes.Camera(173, 97, 140.0, 140.0, 86.0, 48.0, k1=-0.05, k2=0.01, R=R, t=t)
    return sc, cam


@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_forward_does_not_depend_on_threads(orc, which):
    sc, cam = _scene() if which == "tiny" else _mid_scene()
    ref = orc.forward(sc.xyz, sc.feat, cam, 4, 0.01, 1e-3, threads=1)
    assert np.count_nonzero(ref.cnt) > 100
    for t in (2, 3, 8, 0, 64):
        f = orc.forward(sc.xyz, sc.feat, cam, 4, 0.01, 1e-3, threads=t)
        for name in ("keys", "cnt", "img", "pix", "z"):
            assert np.array_equal(getattr(f, name), getattr(ref, name)), (t, name)
    k = orc.keys_counts(sc.xyz, cam, 4, threads=0)
    assert np.array_equal(k.keys, ref.keys) and np.array_equal(k.cnt, ref.cnt)


@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_backward_does_not_depend_on_threads(orc, which):
    sc, cam = _scene() if which == "tiny" else _mid_scene()
    f = orc.forward(sc.xyz, sc.feat, cam, 4, 0.01, 1e-3)
    G = np.concatenate([g.ravel() for g in scenes.upstream_grad(cam.w, cam.h, 4, sc.c, 5)]).astype(np.float64)
    ref = orc.backward(f, sc.xyz, sc.feat, cam, G, 0.01, threads=1)
    assert np.abs(ref.dpose).max() > 0
    for t in (2, 5, 0):
        b = orc.backward(f, sc.xyz, sc.feat, cam, G, 0.01, threads=t)
        for name in ("dfeat", "dxyz", "gu", "gv"):
            assert np.array_equal(getattr(b, name), getattr(ref, name)), (t, name)
        for name in ("dpose", "dintr"):
            got, want, scale = getattr(b, name), getattr(ref, name), getattr(ref, name + "_abs")
            assert np.all(np.abs(got - want) <= 1e-12 * scale), (t, name, got - want)
        assert np.allclose(b.dpose_abs, ref.dpose_abs, rtol=1e-12, atol=0)


def test_sampled_backward_rows_and_sums(orc):
    sc, cam = _mid_scene()
    f = orc.forward(sc.xyz, sc.feat, cam, 4, 0.01, 1e-3)
    G = np.concatenate([g.ravel() for g in scenes.upstream_grad(cam.w, cam.h, 4, sc.c, 6)]).astype(np.float64)
    full = orc.backward(f, sc.xyz, sc.feat, cam, G, 0.01, threads=0)
    rng = np.random.default_rng(4)
    perm = rng.permutation(sc.n)
    parts = [np.sort(perm[:20_000]), np.sort(perm[20_000:45_000]), np.sort(perm[45_000:])]
    pose = np.zeros(6)
    intr = np.zeros(6)
    for s in parts:
        b = orc.backward(f, sc.xyz, sc.feat, cam, G, 0.01, threads=3, sample=s)
        for name in ("dfeat", "dxyz", "gu", "gv"):
            got, want = getattr(b, name), getattr(full, name)
            assert np.array_equal(got[s], want[s]), name
            rest = np.ones(sc.n, bool)
            rest[s] = False
            assert not got[rest].any(), name
        pose += b.dpose
        intr += b.dintr
    assert np.all(np.abs(pose - full.dpose) <= 1e-12 * full.dpose_abs)
    assert np.all(np.abs(intr - full.dintr) <= 1e-12 * full.dintr_abs)
    with pytest.raises(IndexError):
        orc.backward(f, sc.xyz, sc.feat, cam, G, 0.01, sample=np.array([sc.n]))


def test_forward_options_do_not_depend_on_threads(orc):
    """The same with every forward option on: an environment map for the
    empty pixels, stochastic discarding, normal culling and log descriptors."""
    sc, cam = _mid_scene()
    rng = np.random.default_rng(8)
    env = 0.5 + 0.1 * rng.standard_normal((sc.c, 16, 32))
    radius = np.full(sc.n, 0.02, np.float32)
    beta = rng.random(sc.n).astype(np.float32)
    kw = dict(normals=sc.normals, radius=radius, beta=beta, gamma=1.5, log_desc=True, env=env)
    ref = orc.forward(sc.xyz, 0.1 * sc.feat, cam, 4, 0.01, 1e-3, threads=1, **kw)
    assert np.count_nonzero(ref.cnt) > 100 and np.count_nonzero(ref.cnt == 0) > 100
    for t in (3, 0):
        f = orc.forward(sc.xyz, 0.1 * sc.feat, cam, 4, 0.01, 1e-3, threads=t, **kw)
        for name in ("keys", "cnt", "img", "pix", "z"):
            assert np.array_equal(getattr(f, name), getattr(ref, name)), (t, name)
