"""Pins of the oracle's depth test, blending and approximate spatial gradient
(Sec. 3.1: Eq. depthtest, Eq. blend, Eqs. induce / gradp / spatialderiv)
against a hand-worked example, a list-based brute force, the exact
shift-and-rerender change, invariances and special cases.  CPU only."""
import os

import numpy as np
import pytest

from scenes import Camera, tiny_spheres

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_example_1d.txt")


def pixel_camera(w, h):
    """fx = fy = 1, principal point 0, R = I, t = 0: world (u z, v z, z) lands at (u, v)."""
    return Camera(w, h, 1.0, 1.0, 0.0, 0.0, R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32))


def pixel_points(uv, z):
    uv = np.asarray(uv, np.float64)
    z = np.asarray(z, np.float32)
    return np.stack([uv[:, 0] * z, uv[:, 1] * z, z], axis=1).astype(np.float32)


def _golden():
    rows = {}
    pts = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, *vals = line.split()
        if k == "point":
            pts.append((vals[0], float(vals[1]), float(vals[2]), float(vals[3])))
        else:
            rows[k] = np.array([float(v) for v in vals])
    return pts, rows


def test_hand_example(orc):
    pts, rows = _golden()
    cam = pixel_camera(4, 1)
    xyz = pixel_points([(p[1], 0.0) for p in pts], [p[2] for p in pts])
    feat = np.array([[p[3]] for p in pts])
    f = orc.forward(xyz, feat, cam, levels=1, alpha=0.01)
    assert np.array_equal(f.img, rows["image"])
    assert np.array_equal(f.cnt, rows["count"].astype(np.uint32))
    b = orc.backward(f, xyz, feat, cam, rows["grad"], alpha=0.01)
    assert np.allclose(b.dfeat.ravel(), rows["dtau"], rtol=0, atol=1e-15)
    assert np.allclose(b.gu.ravel(), rows["g_u"], rtol=0, atol=1e-15)
    assert np.allclose(b.gv.ravel(), rows["g_v"], rtol=0, atol=1e-15)
    # variant: D at z = 1.008 -> the fuzzy-equal case on both sides
    xyz[3] = pixel_points([(2.0, 0.0)], [rows["variant_D_z"][0]])[0]
    f = orc.forward(xyz, feat, cam, levels=1, alpha=0.01)
    assert np.array_equal(f.img, rows["image"])
    b = orc.backward(f, xyz, feat, cam, rows["grad"], alpha=0.01)
    assert np.allclose(b.gu.ravel(), rows["variant_g_u"], rtol=0, atol=1e-12)


def _random_pixel_scene(seed, n=48, w=8, h=6, c=3):
    """Points on a small image with clustered, near-equal and exactly equal
    depths, so every case of Eq. spatialderiv and the index tie-break occur."""
    rng = np.random.default_rng(seed)
    pu = rng.integers(0, w, n)
    pv = rng.integers(0, h, n)
    jitter = rng.uniform(-0.4, 0.4, size=(n, 2))
    base = np.float32(rng.choice([1.0, 1.5, 2.0], size=n))
    step = rng.choice([0.0, 0.0, 0.004, 0.0099, 0.0101, 0.02, 0.3], size=n)
    z = (base * (1 + step)).astype(np.float32)
    xyz = pixel_points(np.stack([pu + jitter[:, 0], pv + jitter[:, 1]], 1), z)
    feat = rng.normal(size=(n, c))
    return xyz, feat, pixel_camera(w, h)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("all_projected", [False, True])
def test_oracle_equals_list_bruteforce(orc, seed, all_projected):
    levels = 3
    xyz, feat, cam = _random_pixel_scene(seed)
    bg = np.array([0.25, -0.5, 1.0])
    f = orc.forward(xyz, feat, cam, levels=levels, background=bg)
    G = np.random.default_rng(100 + seed).normal(size=f.img.shape)
    b = orc.backward(f, xyz, feat, cam, G, background=bg, all_projected=all_projected)
    G_layers = orc.split_layers(G, cam.w, cam.h, levels, feat.shape[1])
    layers, dfeat, gu, gv = orc.bruteforce_spatial(f.pix.tolist(), f.z, feat, G_layers, cam.w, cam.h,
                                                   levels, background=bg, all_projected=all_projected)
    for l, L in enumerate(layers):
        keys = np.array([np.iinfo(np.uint64).max if k is None else k for k in L["key"]], np.uint64)
        assert np.array_equal(f.layer_keys()[l].ravel(), keys)
        assert np.array_equal(f.layer_cnt()[l].ravel(), np.array([len(m) for m in L["lam"]]))
        assert np.allclose(f.layer_img()[l], L["I"], rtol=0, atol=1e-13)
    assert np.allclose(b.dfeat, dfeat, rtol=0, atol=1e-12)
    assert np.allclose(b.gu, gu, rtol=0, atol=1e-12)
    assert np.allclose(b.gv, gv, rtol=0, atol=1e-12)


def test_spatial_rule_vs_shift_and_rerender(orc):
    """Eq. spatialderiv approximates the exact change at the target pixel.
    Cases 1-3 (empty, behind, in front) are exact; the fuzzy-equal case is
    exact when no target point drops out of the fuzzy band because the
    shifted point becomes the new minimum."""
    from oracle import bruteforce as bf
    a1 = np.float32(np.float32(1.0) + np.float32(0.01))
    seen = {1: 0, 2: 0, 3: 0, 4: 0}
    for seed in range(8):
        xyz, feat, cam = _random_pixel_scene(seed, n=40, w=6, h=5)
        f = orc.forward(xyz, feat, cam, levels=1)
        pix = f.pix.tolist()
        layer = bf.bruteforce_render(pix, f.z, feat, cam.w, cam.h, 1)[0]
        for i in range(len(pix)):
            p = pix[i][0]
            if p < 0 or i not in layer["lam"][p]:
                continue
            pu, pv = p % cam.w, p // cam.w
            for qu, qv in ((pu + 1, pv), (pu - 1, pv), (pu, pv + 1), (pu, pv - 1)):
                if not (0 <= qu < cam.w and 0 <= qv < cam.h):
                    continue
                q = qv * cam.w + qu
                case, d_rule = bf.induced_change(layer, i, f.z[i], feat[i], q)
                d_exact = bf.shift_rerender(pix, f.z, feat, cam.w, cam.h, 1, 0, i, q)
                if case == 4:
                    zi, mz = np.float32(f.z[i]), layer["minz"][q]
                    lo, hi = np.float32(zi * a1), np.float32(mz * a1)
                    drops = any(lo < np.float32(f.z[j]) <= hi for j in layer["lam"][q])
                    if zi < mz and drops:
                        continue
                seen[case] += 1
                assert np.allclose(d_rule, d_exact, rtol=0, atol=1e-12), (case, d_rule, d_exact)
    assert all(v > 0 for v in seen.values()), seen


def _small_sphere_view(n=3000, seed=11):
    sc = tiny_spheres(n, 4, seed=seed)
    cam = Camera(64, 48, 51.25, 51.25, 32.0, 24.0, k1=0.01,
                 R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 2], np.float32))
    return sc, cam


def test_point_order_invariance(orc):
    sc, cam = _small_sphere_view()
    f = orc.forward(sc.xyz, sc.feat, cam)
    G = np.random.default_rng(3).normal(size=f.img.shape)
    b = orc.backward(f, sc.xyz, sc.feat, cam, G)
    perm = np.random.default_rng(4).permutation(sc.n)
    fp = orc.forward(sc.xyz[perm], sc.feat[perm], cam)
    bp = orc.backward(fp, sc.xyz[perm], sc.feat[perm], cam, G)
    # depth half of every key is identical; the index half maps through perm
    assert np.array_equal(f.keys >> np.uint64(32), fp.keys >> np.uint64(32))
    hit = fp.keys != np.iinfo(np.uint64).max
    idx_p = (fp.keys[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    idx = (f.keys[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    z = f.z
    # where the nearest depth is unique the same point wins; on exact ties
    # the winner is the smallest index of each order, at the same depth
    same = perm[idx_p] == idx
    assert np.all(z[perm[idx_p]] == z[idx])
    assert same.mean() > 0.99
    assert np.array_equal(f.cnt, fp.cnt)
    assert np.allclose(f.img, fp.img, rtol=0, atol=1e-12)
    assert np.allclose(b.dfeat[perm], bp.dfeat, rtol=0, atol=1e-12)
    assert np.allclose(b.dxyz[perm], bp.dxyz, rtol=0, atol=1e-9)
    assert np.allclose(b.dpose, bp.dpose, rtol=1e-9, atol=1e-9 * b.dpose_abs.max())
    assert np.allclose(b.dintr, bp.dintr, rtol=1e-9, atol=1e-9 * b.dintr_abs.max())


def test_alpha_zero_is_a_plain_zbuffer(orc):
    sc, cam = _small_sphere_view()
    f = orc.forward(sc.xyz, sc.feat, cam, alpha=0.0)
    for l in range(4):
        hl, wl = cam.h >> l, cam.w >> l
        off = sum((cam.w >> k) * (cam.h >> k) for k in range(l))
        p = f.pix[:, l]
        ok = p >= 0
        # nearest point per pixel by sorting (pixel, depth, index)
        order = np.lexsort((np.arange(sc.n)[ok], f.z[ok], p[ok]))
        pp, ii = p[ok][order], np.arange(sc.n)[ok][order]
        first = np.r_[True, pp[1:] != pp[:-1]]
        want = np.full(hl * wl, -1)
        want[pp[first]] = ii[first]
        got = f.keys[off:off + hl * wl]
        empty = got == np.iinfo(np.uint64).max
        assert np.array_equal(empty, want < 0)
        assert np.array_equal((got[~empty] & np.uint64(0xFFFFFFFF)).astype(np.int64), want[~empty])
        cnt = f.cnt[off:off + hl * wl]
        img = f.layer_img()[l].reshape(sc.c, -1)
        zmin = f.z[want[~empty]]
        ties = np.array([np.sum((p == q) & (f.z == zq)) for q, zq in zip(np.nonzero(~empty)[0], zmin)])
        assert np.array_equal(cnt[~empty], ties)
        single = ties == 1
        assert np.allclose(img[:, ~empty][:, single], sc.feat[want[~empty][single]].T, rtol=0, atol=0)


def test_distinct_pixels(orc):
    rng = np.random.default_rng(8)
    w, h = 12, 9
    cells = rng.permutation(w * h)[:40]
    xyz = pixel_points(np.stack([cells % w, cells // w], 1), rng.uniform(1, 3, 40))
    feat = rng.normal(size=(40, 2))
    cam = pixel_camera(w, h)
    f = orc.forward(xyz, feat, cam, levels=1)
    img = f.img.reshape(2, -1)
    assert np.array_equal(img[:, cells], feat.T)
    assert np.array_equal(f.cnt[cells], np.ones(40, np.uint32))
    G = rng.normal(size=f.img.shape)
    b = orc.backward(f, xyz, feat, cam, G)
    assert np.array_equal(b.dfeat, G.reshape(2, -1)[:, cells].T)


@pytest.mark.parametrize("bg", [None, (0.5, -1.0)])
def test_single_point_is_a_central_difference(orc, bg):
    w, h = 7, 5
    cam = pixel_camera(w, h)
    xyz = pixel_points([(3.2, 2.1)], [1.7])
    tau = np.array([[0.7, -1.3]])
    f = orc.forward(xyz, tau, cam, levels=1, background=bg)
    G = np.random.default_rng(9).normal(size=f.img.shape)
    b = orc.backward(f, xyz, tau, cam, G, background=bg)
    Gi = G.reshape(2, h, w)
    d = tau[0] - (np.zeros(2) if bg is None else np.array(bg))
    assert np.isclose(b.gu[0, 0], 0.5 * (Gi[:, 2, 4] @ d - Gi[:, 2, 2] @ d), rtol=0, atol=1e-14)
    assert np.isclose(b.gv[0, 0], 0.5 * (Gi[:, 3, 3] @ d - Gi[:, 1, 3] @ d), rtol=0, atol=1e-14)


def test_feature_gradient_is_exact_for_linear_blend(orc):
    """I is linear in tau, so any finite difference of L = <G, I> is exact."""
    sc, cam = _small_sphere_view(n=1500)
    f = orc.forward(sc.xyz, sc.feat, cam)
    G = np.random.default_rng(12).normal(size=f.img.shape)
    b = orc.backward(f, sc.xyz, sc.feat, cam, G)
    rng = np.random.default_rng(13)
    base = G @ f.img
    for i in rng.choice(sc.n, 25, replace=False):
        for ch in range(sc.c):
            fe = sc.feat.astype(np.float64).copy()
            fe[i, ch] += 1.0
            fp = orc.forward(sc.xyz, fe, cam)
            assert np.isclose(G @ fp.img - base, b.dfeat[i, ch], rtol=1e-9, atol=1e-9)


def test_normal_culling_literal(orc):
    # keep iff (R n)^T (R x + t) > 0 (Eq. normalculling as printed)
    cam = pixel_camera(4, 1)
    xyz = pixel_points([(1.0, 0.0), (2.0, 0.0)], [1.0, 1.0])
    nrm = np.array([[0, 0, 1.0], [0, 0, -1.0]], np.float32)
    f = orc.forward(xyz, np.ones((2, 1)), cam, levels=1, normals=nrm)
    assert f.pix[:, 0].tolist() == [1, -1]


def test_log_descriptors(orc):
    """Logarithmic descriptors (Sec. 3.2) are blended as exp(tau): the render
    of log(F) with conversion equals the render of F, and dL/dtau is the
    linear gradient times exp(tau) -- checked by central differences."""
    sc, cam = _small_sphere_view(n=1200)
    F = np.exp(np.random.default_rng(5).normal(scale=0.7, size=(sc.n, sc.c)))
    a = orc.forward(sc.xyz, np.log(F), cam, log_desc=True)
    b = orc.forward(sc.xyz, F, cam)
    assert np.array_equal(a.keys, b.keys) and np.allclose(a.img, b.img, rtol=1e-12, atol=1e-12)
    G = np.random.default_rng(6).normal(size=a.img.shape)
    ga = orc.backward(a, sc.xyz, np.log(F), cam, G, log_desc=True)
    gb = orc.backward(b, sc.xyz, F, cam, G)
    assert np.allclose(ga.dfeat, gb.dfeat * F, rtol=1e-12, atol=1e-12)
    assert np.allclose(ga.dxyz, gb.dxyz, rtol=1e-9, atol=1e-9)
    tau = np.log(F)
    rng = np.random.default_rng(7)
    for i in rng.choice(np.nonzero(np.abs(ga.dfeat).sum(1))[0], 10, replace=False):
        for ch in range(sc.c):
            tp, tm = tau.copy(), tau.copy()
            tp[i, ch] += 1e-6
            tm[i, ch] -= 1e-6
            fd = (G @ orc.forward(sc.xyz, tp, cam, log_desc=True).img - G @ orc.forward(sc.xyz, tm, cam, log_desc=True).img) / 2e-6
            assert np.isclose(fd, ga.dfeat[i, ch], rtol=1e-5, atol=1e-7)


def test_keys_counts_equal_the_full_forward(orc):
    # the descriptor-free forward used for the largest clouds is the same
    # computation as the full forward, up to the blend
    sc = tiny_spheres(4000, 4, seed=71)
    cam = Camera(96, 64, 80.0, 80.0, 48.0, 32.0, k1=0.02, R=np.eye(3, dtype=np.float32),
                 t=np.array([-0.5, -0.4, 2.5], np.float32))
    f = orc.forward(sc.xyz, sc.feat, cam)
    k = orc.keys_counts(sc.xyz, cam)
    assert np.array_equal(f.keys, k.keys) and np.array_equal(f.cnt, k.cnt)
    assert np.array_equal(f.pix, k.pix) and np.array_equal(f.z, k.z)
