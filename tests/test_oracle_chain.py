"""Pin of the oracle's chain rule (Eq. partial, Eq. tangent): the position,
pose and intrinsics gradients against central finite differences.

Finite differences of the rendered image itself are zero almost everywhere
(Eq. round makes it piecewise constant), so they cannot check position
gradients.  Instead the per-(point, layer) pixel gradients (g_u, g_v) that the
oracle produced are frozen and the surrogate

    S(theta) = sum_i sum_l 2^-l (g_u[i,l] u0_i(theta) + g_v[i,l] v0_i(theta))

is differenced with respect to positions, the left pose increment
exp(xi) (R, t) (the SE(3) exponential taken from scipy's matrix exponential,
independent of the oracle) and the intrinsics.  CPU only."""
import numpy as np
import pytest
from scipy.linalg import expm

from scenes import Camera, tiny_spheres


def _hat(xi):
    nu, om = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]]
    M[:3, 3] = nu
    return M


def _scene(model=0):
    sc = tiny_spheres(2500, 3, seed=21)
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec([0.05, -0.1, 0.02]).as_matrix().astype(np.float32)
    if model == 1:  # a wide fisheye close to the spheres
        cam = Camera(96, 80, 30.0, 30.0, 48.5, 40.5, k1=0.05, k2=-0.02, k3=0.004, R=R,
                     t=np.array([-0.4, -0.3, 0.9], np.float32), model=1)
    else:
        cam = Camera(80, 60, 64.0, 62.0, 40.5, 29.5, k1=0.05, k2=-0.02, k3=0.004, p1=0.003, p2=-0.002,
                     R=R, t=np.array([-0.4, -0.3, 2.2], np.float32))
    return sc, cam


@pytest.fixture(scope="module", params=[0, 1], ids=["pinhole", "fisheye"])
def grads(orc, request):
    sc, cam = _scene(request.param)
    f = orc.forward(sc.xyz, sc.feat, cam)
    G = np.random.default_rng(22).normal(size=f.img.shape)
    b = orc.backward(f, sc.xyz, sc.feat, cam, G)
    wgt = np.ldexp(1.0, -np.arange(f.levels))
    wu = (b.gu * wgt).sum(1)
    wv = (b.gv * wgt).sum(1)
    return sc, cam, b, wu, wv


def _k9(cam):
    return np.array([np.float64(np.float32(getattr(cam, k))) for k in
                     ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")])


def _surrogate(orc, k9, R, t, xyz, wu, wv, model=0):
    X = xyz @ R.T + t
    uv = orc.camera_f64_many(k9, X, model)
    return float(wu @ uv[:, 0] + wv @ uv[:, 1])


def test_nontrivial(grads):
    sc, cam, b, wu, wv = grads
    assert np.count_nonzero(wu) > 200 and np.abs(b.dpose).max() > 0


def test_position_gradient(orc, grads):
    sc, cam, b, wu, wv = grads
    k9 = _k9(cam)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    xyz = sc.xyz.astype(np.float64)
    idx = np.nonzero(wu)[0][:40]
    for i in idx:
        for k in range(3):
            h = 1e-6
            xp, xm = xyz[i:i + 1].copy(), xyz[i:i + 1].copy()
            xp[0, k] += h
            xm[0, k] -= h
            fd = (_surrogate(orc, k9, R, t, xp, wu[i:i + 1], wv[i:i + 1], cam.model)
                  - _surrogate(orc, k9, R, t, xm, wu[i:i + 1], wv[i:i + 1], cam.model)) / (2 * h)
            assert np.isclose(fd, b.dxyz[i, k], rtol=1e-6, atol=1e-6 * np.abs(b.dxyz[i]).max())


def test_pose_gradient_left_increment(orc, grads):
    sc, cam, b, wu, wv = grads
    k9 = _k9(cam)
    T = np.eye(4)
    T[:3, :3] = cam.R.astype(np.float64)
    T[:3, 3] = cam.t.astype(np.float64)
    xyz = sc.xyz.astype(np.float64)
    for k in range(6):
        h = 1e-6
        vals = []
        for s in (+1, -1):
            xi = np.zeros(6)
            xi[k] = s * h
            Tp = expm(_hat(xi)) @ T
            vals.append(_surrogate(orc, k9, Tp[:3, :3], Tp[:3, 3], xyz, wu, wv, cam.model))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - b.dpose[k]) <= 1e-6 * b.dpose_abs[k], (k, fd, b.dpose[k])


def test_intrinsics_gradient(orc, grads):
    sc, cam, b, wu, wv = grads
    k9 = _k9(cam)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    xyz = sc.xyz.astype(np.float64)
    for k in range(6):
        h = 1e-6 * max(1.0, abs(k9[k]))
        kp, km = k9.copy(), k9.copy()
        kp[k] += h
        km[k] -= h
        fd = (_surrogate(orc, kp, R, t, xyz, wu, wv, cam.model)
              - _surrogate(orc, km, R, t, xyz, wu, wv, cam.model)) / (2 * h)
        assert abs(fd - b.dintr[k]) <= 1e-6 * b.dintr_abs[k], (k, fd, b.dintr[k])
