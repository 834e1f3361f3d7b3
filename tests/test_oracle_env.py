"""Pins of the oracle's environment map (Sec. 3.1: empty pixels show a learned
spherical map sampled along the pixel's ray): the inverse camera against the
forward camera, the equirectangular lookup against directions built from
texel coordinates, the forward's use of it, and dL/dE against the forward's
linearity in E.  CPU only."""
import numpy as np
import pytest

from scenes import Camera, env_map, tiny_spheres


def _dir_from_texel(ue, ve, ew, eh):
    """World direction whose longitude / colatitude put it at texel
    coordinates (ue, ve) (texel centres at integers)."""
    phi = (ue + 0.5) / ew * 2 * np.pi - np.pi
    theta = (ve + 0.5) / eh * np.pi
    return np.array([np.sin(theta) * np.sin(phi), np.cos(theta), np.sin(theta) * np.cos(phi)])


def _cams():
    pin = Camera(80, 60, 64.0, 62.0, 40.5, 29.5, k1=0.05, k2=-0.02, k3=0.004, p1=0.003, p2=-0.002)
    fish = Camera(96, 80, 30.0, 30.0, 48.5, 40.5, k1=0.05, k2=-0.02, k3=0.004, model=1)
    return [pin, fish]


@pytest.mark.parametrize("model", [0, 1], ids=["pinhole", "fisheye"])
def test_inverse_camera_inverts_projection(orc, model):
    cam = _cams()[model]
    rng = np.random.default_rng(40 + model)
    # directions within ~35 degrees (pinhole) / ~75 degrees (fisheye) of the axis
    span = 0.7 if model == 0 else 2.5
    X = np.stack([rng.uniform(-span, span, 200), rng.uniform(-span, span, 200), np.ones(200)], axis=1)
    X *= rng.uniform(0.5, 9.0, (200, 1))
    k9 = np.array([np.float64(np.float32(getattr(cam, k))) for k in ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")])
    uv = orc.camera_f64_many(k9, X, model)
    for i in range(200):
        d = orc.camera_inverse(cam, uv[i, 0], uv[i, 1])
        assert np.allclose(d, X[i] / np.linalg.norm(X[i]), rtol=0, atol=1e-12), (i, d)


def test_inverse_camera_principal_point_is_the_axis(orc):
    for cam in _cams():
        d = orc.camera_inverse(cam, np.float32(cam.cx), np.float32(cam.cy))
        assert np.array_equal(d, [0.0, 0.0, 1.0])


def test_env_sample_constant_and_texel_centres(orc):
    rng = np.random.default_rng(41)
    ew, eh, c = 16, 8, 3
    const = np.broadcast_to(np.array([0.25, -1.0, 3.0])[:, None, None], (c, eh, ew))
    E = rng.normal(size=(c, eh, ew))
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        assert np.allclose(orc.env_sample(const, d), [0.25, -1.0, 3.0], rtol=0, atol=1e-15)
    for j in range(eh):
        for i in range(ew):
            s = orc.env_sample(E, _dir_from_texel(float(i), float(j), ew, eh))
            assert np.allclose(s, E[:, j, i], rtol=0, atol=1e-12), (i, j)


def test_env_sample_is_bilinear(orc):
    # a map linear in the texel indices is reproduced exactly between texel
    # centres (away from the longitude seam, inside the colatitude range)
    ew, eh = 24, 12
    i, j = np.meshgrid(np.arange(ew), np.arange(eh))
    E = np.stack([0.3 * i - 0.7 * j, 2.0 + 0.05 * j + 0.0 * i])
    rng = np.random.default_rng(42)
    for _ in range(50):
        ue, ve = rng.uniform(0, ew - 1), rng.uniform(0, eh - 1)
        s = orc.env_sample(E, _dir_from_texel(ue, ve, ew, eh))
        assert np.allclose(s, [0.3 * ue - 0.7 * ve, 2.0 + 0.05 * ve], rtol=0, atol=1e-11)


def test_env_sample_wraps_longitude_and_clamps_colatitude(orc):
    ew, eh = 8, 4
    E = np.arange(ew * eh, dtype=np.float64).reshape(1, eh, ew) ** 1.5
    row = 2
    # just past -pi: a quarter of the way from the last column to the first
    s = orc.env_sample(E, _dir_from_texel(-0.25, float(row), ew, eh))
    assert np.isclose(s[0], 0.25 * E[0, row, ew - 1] + 0.75 * E[0, row, 0], rtol=0, atol=1e-12)
    s = orc.env_sample(E, _dir_from_texel(ew - 0.75, float(row), ew, eh))
    assert np.isclose(s[0], 0.75 * E[0, row, ew - 1] + 0.25 * E[0, row, 0], rtol=0, atol=1e-12)
    # above the first row's centres the first row is used alone
    s = orc.env_sample(E, _dir_from_texel(2.5, -0.3, ew, eh))
    assert np.isclose(s[0], 0.5 * (E[0, 0, 2] + E[0, 0, 3]), rtol=0, atol=1e-12)
    s = orc.env_sample(E, _dir_from_texel(5.0, eh - 0.6, ew, eh))
    assert np.isclose(s[0], E[0, eh - 1, 5], rtol=0, atol=1e-12)


def test_forward_empty_pixels_sample_the_ray(orc):
    # no points: every pixel of every layer is empty.  A camera turned to look
    # along world +x (R's third row = (1, 0, 0)) sees, at the principal point
    # of each layer, the map's texel coordinates (3/4 ew - 1/2, eh/2 - 1/2);
    # at the pixel a quarter turn further (u0 - cx = fx) the longitude is pi/4
    # further round.
    ew, eh = 32, 16
    i, j = np.meshgrid(np.arange(ew), np.arange(eh))
    E = np.stack([0.1 * i + 0.01 * j]).astype(np.float64)
    R = np.array([[0, 0, -1], [0, 1, 0], [1, 0, 0]], np.float32)
    cam = Camera(64, 48, 16.0, 16.0, 32.0, 24.0, R=R, t=np.array([0.3, -0.2, 1.0], np.float32))
    f = orc.forward(np.zeros((0, 3), np.float32), np.zeros((0, 1), np.float32), cam, levels=4, env=E)
    assert not f.cnt.any()
    off = 0
    for l in range(4):
        wl, hl = 64 >> l, 48 >> l
        img = f.img[off:off + wl * hl].reshape(hl, wl)
        ue, ve = 0.75 * ew - 0.5, 0.5 * eh - 0.5
        assert np.isclose(img[24 >> l, 32 >> l], 0.1 * ue + 0.01 * ve, rtol=0, atol=1e-12), l
        if l <= 2:  # u0 = cx + fx = 48 is a pixel centre of layers 0..2
            ue2 = ue + ew / 8.0
            assert np.isclose(img[24 >> l, 48 >> l], 0.1 * ue2 + 0.01 * ve, rtol=0, atol=1e-12), l
        off += wl * hl


def _scene_with_gaps():
    sc = tiny_spheres(3000, 3, seed=43)
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec([0.2, -0.5, 0.1]).as_matrix().astype(np.float32)
    cam = Camera(80, 60, 50.0, 48.0, 40.5, 29.5, k1=0.05, k2=-0.02, p1=0.002, R=R,
                 t=np.array([-0.4, -0.3, 2.6], np.float32))
    return sc, cam


def test_constant_map_equals_background(orc):
    sc, cam = _scene_with_gaps()
    bg = np.array([0.2, -0.4, 0.9])
    const = np.broadcast_to(bg[:, None, None], (3, 8, 16))
    fb = orc.forward(sc.xyz, sc.feat, cam, background=bg)
    fe = orc.forward(sc.xyz, sc.feat, cam, env=const)
    assert 0 < np.count_nonzero(fe.cnt == 0) < fe.cnt.size
    # (the four bilinear weights sum to 1 up to rounding)
    assert np.allclose(fb.img, fe.img, rtol=0, atol=1e-15) and np.array_equal(fb.cnt, fe.cnt)
    G = np.random.default_rng(44).normal(size=fb.img.shape)
    bb = orc.backward(fb, sc.xyz, sc.feat, cam, G, background=bg)
    be = orc.backward(fe, sc.xyz, sc.feat, cam, G, background=bg)
    assert np.allclose(bb.dxyz, be.dxyz, rtol=1e-12, atol=1e-12) and np.array_equal(bb.dfeat, be.dfeat)


def test_env_gradient_is_the_forward_linear_map(orc):
    # for fixed geometry the image is linear in E, so dL/dE[t] of
    # L = <G, img> is exactly L(E + e_t) - L(E)
    sc, cam = _scene_with_gaps()
    E = env_map(3, 8, 16, seed=45).astype(np.float64)
    f = orc.forward(sc.xyz, sc.feat, cam, env=E)
    G = np.random.default_rng(46).normal(size=f.img.shape)
    dE = orc.env_grad(f, cam, G, E.shape)
    assert np.count_nonzero(dE) > 20
    L0 = float(G @ f.img)
    rng = np.random.default_rng(47)
    hit = np.flatnonzero(dE)
    for t in list(rng.choice(hit, 12, replace=False)) + [int(np.flatnonzero(dE == 0)[0])]:
        Ep = E.copy().ravel()
        Ep[t] += 1.0
        L1 = float(G @ orc.forward(sc.xyz, sc.feat, cam, env=Ep.reshape(E.shape)).img)
        assert np.isclose(L1 - L0, dE.ravel()[t], rtol=1e-9, atol=1e-9), t
