"""Pins of the oracle's stochastic point discarding (Sec. 3.1, Eq. discard:
keep iff r_screen / sqrt(1 - beta) > 1 / gamma) and of the world-radius
preprocess (distance to the 4th-nearest point).  CPU only."""
import numpy as np
import pytest

from scenes import Camera, tiny_spheres


def _pixel_cam(w=16, h=16):
    return Camera(w, h, 1.0, 1.0, 0.0, 0.0, R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32))


def test_threshold_with_beta_zero(orc):
    """beta = 0: keep iff gamma * r_screen > 1, r_screen = fx r / (z 2^l).
    With fx = 1, z = 1 and gamma = 1.5 that is r > 2^l / 1.5, by hand."""
    cam = _pixel_cam()
    radii = np.array([0.5, 1.0, 2.0, 3.0, 6.0, 12.0], np.float32)
    n = len(radii)
    xyz = np.stack([np.full(n, 8.2), np.full(n, 8.2), np.ones(n)], 1).astype(np.float32)
    f = orc.forward(xyz, np.ones((n, 1)), cam, levels=4, radius=radii, beta=np.zeros(n, np.float32), gamma=1.5)
    want = np.array([[r > 2.0 ** l / 1.5 for l in range(4)] for r in radii])
    # by hand: 0.5 -> none; 1 -> l0; 2 -> l0,l1; 3 -> l0..l2; 6 -> l0..l3; 12 -> all
    assert want.sum(1).tolist() == [0, 1, 2, 3, 4, 4]
    assert np.array_equal(f.pix >= 0, want)


def test_large_gamma_discards_nothing(orc):
    sc = tiny_spheres(3000, 2, seed=3)
    cam = Camera(64, 48, 51.25, 51.25, 32.0, 24.0, R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 2], np.float32))
    rng = np.random.default_rng(0)
    r = np.full(sc.n, 0.01, np.float32)
    a = orc.forward(sc.xyz, sc.feat, cam)
    b = orc.forward(sc.xyz, sc.feat, cam, radius=r, beta=rng.random(sc.n).astype(np.float32), gamma=1e6)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.cnt, b.cnt) and np.array_equal(a.img, b.img)


def test_kept_fraction_is_the_stated_probability(orc):
    """With beta ~ U[0,1) the keep probability is min(1, (gamma r_screen)^2)."""
    cam = _pixel_cam(64, 64)
    n = 40000
    rng = np.random.default_rng(1)
    xyz = np.stack([rng.uniform(10, 50, n), rng.uniform(10, 50, n), np.ones(n)], 1).astype(np.float32)
    r = np.full(n, 0.4, np.float32)  # gamma r_screen = 0.6, 0.3, 0.15, 0.075
    f = orc.forward(xyz, np.ones((n, 1)), cam, levels=4, radius=r, beta=rng.random(n).astype(np.float32),
                    gamma=1.5)
    for l in range(4):
        p = min(1.0, (1.5 * 0.4 / 2 ** l) ** 2)
        got = (f.pix[:, l] >= 0).mean()
        assert abs(got - p) < 4 * np.sqrt(p * (1 - p) / n) + 1e-4, (l, got, p)
    # a point kept at a coarser layer is kept at every finer layer (r_screen halves per layer)
    kept = f.pix >= 0
    assert np.all(kept[:, 1:] <= kept[:, :-1])


def test_discard_with_list_bruteforce(orc):
    """Discarded (point, layer) pairs neither occlude, blend nor get gradients:
    the list-based brute force on the oracle's pixel table agrees."""
    sc = tiny_spheres(400, 3, seed=9)
    cam = Camera(24, 18, 20.0, 20.0, 12.0, 9.0, R=np.eye(3, dtype=np.float32), t=np.array([-0.5, -0.5, 2.0], np.float32))
    rng = np.random.default_rng(2)
    r = orc.knn_radius(sc.xyz).astype(np.float32)
    beta = rng.random(sc.n).astype(np.float32)
    f = orc.forward(sc.xyz, sc.feat, cam, levels=3, radius=r, beta=beta, gamma=1.5)
    assert (f.pix < 0).sum() > (orc.forward(sc.xyz, sc.feat, cam, levels=3).pix < 0).sum()
    G = rng.normal(size=f.img.shape)
    b = orc.backward(f, sc.xyz, sc.feat, cam, G)
    layers, dfeat, gu, gv = orc.bruteforce_spatial(f.pix.tolist(), f.z, sc.feat.astype(np.float64),
                                                   orc.split_layers(G, cam.w, cam.h, 3, 3), cam.w, cam.h, 3)
    assert np.allclose(b.dfeat, dfeat, atol=1e-12) and np.allclose(b.gu, gu, atol=1e-12)
    assert np.allclose(b.gv, gv, atol=1e-12)
    for l, L in enumerate(layers):
        assert np.array_equal(f.layer_cnt()[l].ravel(), np.array([len(m) for m in L["lam"]]))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_knn_radius_matches_kdtree(orc, seed):
    """The 4th-nearest-point radius (the paper's preprocess) against scipy's
    k-d tree, including duplicated points (distance 0) and a cloud too small
    to have 4 neighbours."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    xyz = rng.normal(size=(700, 3)).astype(np.float32)
    xyz[10:20] = xyz[0]  # duplicates
    want = cKDTree(xyz.astype(np.float64)).query(xyz.astype(np.float64), k=5)[0][:, 4]
    assert np.allclose(orc.knn_radius(xyz, 4), want, rtol=1e-12, atol=1e-12)
    assert np.all(np.isinf(orc.knn_radius(xyz[:4], 4)))
    assert np.isfinite(orc.knn_radius(xyz[:5], 4)).all()
