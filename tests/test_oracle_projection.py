"""Pins of the oracle's projection (Sec. 3.1: P_l = 2^-l C(Rx + t), Eq. round,
Eq. boundscheck) against hand-derived closed forms and independent
finite differences.  CPU only."""
import math
import os

import numpy as np
import pytest

from scenes import Camera

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "projection_closed_form.txt")


def _parse_golden():
    cams, pts = {}, []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        kind, rest = line.split(None, 1)
        if kind == "camera":
            parts = rest.split("|")
            head, R, t = parts[:3]
            model = int(parts[3]) if len(parts) > 3 else 0
            f = head.split()
            name, w, h = f[0], int(f[1]), int(f[2])
            vals = [float(v) for v in f[3:]]
            cams[name] = Camera(w, h, *vals, R=np.array(R.split(), np.float32).reshape(3, 3),
                                t=np.array(t.split(), np.float32), model=model)
        else:
            head, exp, pix = rest.split("|")
            f = head.split()
            name, x = f[0], [float(v) for v in f[1:4]]
            u0, v0, z = (float(v) for v in exp.split())
            layers = [None if p == "none" else tuple(int(q) for q in p.split(",")) for p in pix.split()]
            pts.append((name, x, u0, v0, z, layers))
    return cams, pts


CAMS, POINTS = _parse_golden()


@pytest.mark.parametrize("row", POINTS, ids=lambda r: f"{r[0]}-{r[1]}")
def test_fp32_contract_matches_closed_form(orc, row):
    name, x, u0, v0, z, layers = row
    cam = CAMS[name]
    gu, gv, gz = orc.project_f32(cam, x)
    # the FP32 contract rounds each of ~15 operations once: a few ulps of the exact value
    for got, want in ((gu, u0), (gv, v0), (gz, z)):
        if np.isnan(want):
            continue
        assert abs(float(got) - want) <= 8 * np.spacing(np.float32(abs(want) + 1.0)), (got, want)
    f = orc.forward(np.array([x], np.float32), np.ones((1, 1)), cam, levels=len(layers))
    for l, want in enumerate(layers):
        got = f.pix[0, l]
        assert (None if got < 0 else (got % (cam.w >> l), got // (cam.w >> l))) == want, (l, want)


@pytest.mark.parametrize("row", POINTS, ids=lambda r: f"{r[0]}-{r[1]}")
def test_fp64_camera_matches_closed_form(orc, row):
    name, x, u0, v0, z, _ = row
    cam = CAMS[name]
    if np.isnan(u0):
        return
    X = cam.R.astype(np.float64) @ np.array(x) + cam.t.astype(np.float64)
    k9 = [cam.fx, cam.fy, cam.cx, cam.cy, cam.k1, cam.k2, cam.k3, cam.p1, cam.p2]
    cam_f64 = orc.camera_fisheye_f64 if cam.model == 1 else orc.camera_f64
    uv = cam_f64(np.array(k9, np.float64), X)
    # exact decimal inputs in FP64: the closed form to FP64 round-off
    assert abs(uv[0] - u0) <= 1e-12 * abs(u0) and abs(uv[1] - v0) <= 1e-12 * abs(v0)
    k9d = [np.float64(np.float32(v)) for v in k9]
    uv2, Xo, _, _ = orc.project_jac_f64(cam, x)
    assert np.allclose(uv2, cam_f64(np.array(k9d), Xo), rtol=0, atol=1e-12)


def test_rounding_half_to_even_and_bounds(orc):
    # Eq. round: nearest integer, ties to even (reading of an unstated tie rule)
    assert orc.pixel(2.5, 0.0, 0, 8, 1) == (2, 0)
    assert orc.pixel(3.5, 0.0, 0, 8, 1) == (4, 0)
    assert orc.pixel(5.0, 0.0, 1, 8, 2) == (2, 0)   # 2.5 at layer 1
    assert orc.pixel(7.0, 0.0, 1, 16, 2) == (4, 0)  # 3.5 at layer 1
    # Eq. boundscheck: p in [0, w[ x [0, h[
    assert orc.pixel(-0.5, 0.0, 0, 4, 1) == (0, 0)  # rounds to -0 -> 0
    assert orc.pixel(-0.6, 0.0, 0, 4, 1) is None
    assert orc.pixel(3.49, 0.0, 0, 4, 1) == (3, 0)
    assert orc.pixel(3.5, 0.0, 0, 4, 1) is None     # rounds to 4 = w
    assert orc.pixel(0.0, 0.6, 0, 4, 1) is None     # rounds to 1 = h
    for bad in (math.nan, math.inf, -math.inf, 1e30, -1e30):
        assert orc.pixel(bad, 0.0, 0, 4, 1) is None
        assert orc.pixel(0.0, bad, 0, 4, 1) is None


def test_layers_round_independently(orc):
    # each layer rounds its own coordinate 2^-l u0 (not the layer-0 pixel)
    assert [orc.pixel(158.757, 10.0, l, 256, 256)[0] for l in range(4)] == [159, 79, 40, 20]
    # layer sizes floor: a 7-wide image has layers 7, 3, 1
    assert orc.pixel(6.0, 0.0, 0, 7, 4) == (6, 0)
    assert orc.pixel(6.0, 0.0, 1, 7, 4) is None     # 3.0 >= w_1 = 3
    assert orc.pixel(4.0, 0.0, 2, 7, 4) is None     # 1.0 >= w_2 = 1


def test_pinhole_special_case(orc):
    # no distortion: u0 = fx X/Z + cx, the textbook pinhole
    cam = Camera(640, 480, 500.0, 400.0, 320.0, 240.0)
    for x in [(0.5, -0.25, 4.0), (-1.0, 0.75, 2.0), (2.0, 2.0, 8.0)]:
        u, v, z = orc.project_f32(cam, x)
        assert u == np.float32(320.0 + 500.0 * x[0] / x[2])
        assert v == np.float32(240.0 + 400.0 * x[1] / x[2])
        assert z == np.float32(x[2])


def _random_cam(rng, model=0):
    return Camera(320, 240, rng.uniform(200, 400), rng.uniform(200, 400), rng.uniform(140, 180),
                  rng.uniform(100, 140), k1=rng.uniform(-0.2, 0.2), k2=rng.uniform(-0.05, 0.05),
                  k3=rng.uniform(-0.01, 0.01), p1=0.0 if model else rng.uniform(-0.01, 0.01),
                  p2=0.0 if model else rng.uniform(-0.01, 0.01),
                  R=_rot(rng), t=rng.normal(size=3).astype(np.float32) + np.array([0, 0, 5], np.float32),
                  model=model)


def _rot(rng):
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(rng.normal(scale=0.3, size=3)).as_matrix().astype(np.float32)


@pytest.mark.parametrize("model", [0, 1])
def test_fp32_and_fp64_projection_agree(orc, model):
    rng = np.random.default_rng(5 + model)
    for _ in range(200):
        cam = _random_cam(rng, model)
        x = rng.normal(size=3).astype(np.float32)
        u, v, z = orc.project_f32(cam, x)
        uv, X, _, _ = orc.project_jac_f64(cam, x)
        assert abs(u - uv[0]) < 2e-4 * (1 + abs(uv[0])) and abs(v - uv[1]) < 2e-4 * (1 + abs(uv[1]))
        depth = np.linalg.norm(X) if model else X[2]
        assert abs(z - depth) < 1e-5 * (1 + abs(depth))


@pytest.mark.parametrize("model", [0, 1])
def test_jacobians_match_finite_differences(orc, model):
    """d(u0,v0)/dX and d(u0,v0)/d(fx,fy,cx,cy,k1,k2) vs central differences
    of the FP64 camera model with every distortion coefficient non-zero
    (pinhole + Brown-Conrady, and the stereographic fisheye)."""
    rng = np.random.default_rng(6 + model)
    cam_f64 = orc.camera_fisheye_f64 if model == 1 else orc.camera_f64
    for _ in range(50):
        cam = _random_cam(rng, model)
        x = rng.normal(size=3).astype(np.float32) * (3.0 if model else 1.0)
        uv, X, JX, JK = orc.project_jac_f64(cam, x)
        k9 = np.array([np.float64(np.float32(getattr(cam, k))) for k in
                       ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")])
        for k in range(3):
            h = 1e-6 * max(1.0, abs(X[k]))
            Xp, Xm = X.copy(), X.copy()
            Xp[k] += h
            Xm[k] -= h
            fd = (cam_f64(k9, Xp) - cam_f64(k9, Xm)) / (2 * h)
            assert np.allclose(fd, JX[:, k], rtol=1e-6, atol=1e-6 * np.abs(JX).max())
        for k in range(6):
            h = 1e-6 * max(1.0, abs(k9[k]))
            kp, km = k9.copy(), k9.copy()
            kp[k] += h
            km[k] -= h
            fd = (cam_f64(kp, X) - cam_f64(km, X)) / (2 * h)
            assert np.allclose(fd, JK[:, k], rtol=1e-6, atol=1e-7 * max(1.0, np.abs(JK[:, k]).max()))


def _nearest(pix, depth):
    """pixel -> index of its nearest point (ties to the smaller index)."""
    sel = np.flatnonzero(pix >= 0)
    order = np.lexsort((sel, depth[sel], pix[sel]))
    p = pix[sel][order]
    first = np.r_[True, p[1:] != p[:-1]]
    return dict(zip(p[first].tolist(), sel[order][first].tolist()))


@pytest.mark.parametrize("which", ["tiny", "single_view_subsample"])
def test_fp64_projection_statistic(orc, which):
    """A statistic, not a gate: how often the FP32 projection contract puts a
    (point, layer) pair in another pixel, or another point in front at a
    pixel, than an FP64 projection of the same inputs would.  Both are rare
    (the points within an FP32 rounding of a pixel edge or of a depth tie)."""
    import scenes
    if which == "tiny":
        sc, cams = scenes.config(1)
    else:
        sc, cams = scenes.config(2, n=200_000)
    cam = cams[0]
    levels = 4
    f = orc.keys_counts(sc.xyz, cam, levels)
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    X = sc.xyz.astype(np.float64) @ R.T + t
    k9 = np.array([np.float64(np.float32(getattr(cam, k))) for k in ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")])
    uv = orc.camera_f64_many(k9, X, 0)
    z = X[:, 2]
    moved = 0
    pairs = 0
    winners_differ = 0
    pixels = 0
    for l in range(levels):
        wl, hl = cam.w >> l, cam.h >> l
        pu = np.rint(uv[:, 0] / 2 ** l)
        pv = np.rint(uv[:, 1] / 2 ** l)
        ok = (z > 1e-3) & (pu >= 0) & (pu < wl) & (pv >= 0) & (pv < hl)
        p64 = np.where(ok, pv * wl + pu, -1).astype(np.int64)
        p32 = f.pix[:, l].astype(np.int64)
        both = (p32 >= 0) | (p64 >= 0)
        pairs += int(both.sum())
        moved += int((p32 != p64)[both].sum())
        w32 = _nearest(p32, f.z.astype(np.float64))
        w64 = _nearest(p64, z)
        common = set(w32) & set(w64)
        pixels += len(common)
        winners_differ += sum(1 for p in common if w32[p] != w64[p])
    frac_moved = moved / max(pairs, 1)
    frac_winner = winners_differ / max(pixels, 1)
    print(f"\n{which}: pairs in another pixel {frac_moved:.2e}, pixels with another nearest point {frac_winner:.2e}")
    assert frac_moved < 1e-3 and frac_winner < 1e-3
