"""The tangent-space pose update (Eq. tangent) behind the C ABI:
adop_pose_apply_tangent against scipy's matrix exponential of the twist,
composed with the pose in FP64.  Host code only (no GPU)."""
import ctypes as ct

import numpy as np
import pytest
from scipy.linalg import expm


def _hat(xi):
    nu, om = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]]
    M[:3, 3] = nu
    return M


def _random_pose(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    return R.astype(np.float32), rng.normal(size=3).astype(np.float32) * 5


@pytest.fixture(scope="module")
def adop():
    import paper_2110_06635_gb300 as adop
    adop.build()
    adop.load()
    return adop


def test_pose_update_matches_matrix_exponential(adop):
    from paper_2110_06635_gb300._abi import adop_pose_apply_tangent
    rng = np.random.default_rng(0)
    for scale in (1e-10, 1e-4, 0.1, 0.9, 1.0, 1.1, 2.5, 3.1):
        for _ in range(20):
            xi = rng.normal(size=6) * scale
            R, t = _random_pose(rng)
            T = np.eye(4)
            T[:3, :3], T[:3, 3] = R, t
            ref = expm(_hat(xi)) @ T
            R1, t1 = adop_pose_apply_tangent(xi, R, t)
            # one FP32 rounding of an FP64 result: within 1 ulp of |entries| <= 1 (R) and of |t'|
            assert np.max(np.abs(R1 - ref[:3, :3])) <= 1.2e-7, (scale, R1 - ref[:3, :3])
            tol = 1.2e-7 * max(1.0, float(np.max(np.abs(ref[:3, 3]))))
            assert np.max(np.abs(t1 - ref[:3, 3])) <= tol, (scale, t1 - ref[:3, 3])


def test_zero_tangent_is_identity(adop):
    from paper_2110_06635_gb300._abi import adop_pose_apply_tangent
    R, t = _random_pose(np.random.default_rng(5))
    R1, t1 = adop_pose_apply_tangent(np.zeros(6), R, t)
    assert np.array_equal(R1, R) and np.array_equal(t1, t)


def test_batched_call_and_errors(adop):
    from paper_2110_06635_gb300 import _abi as A
    lib = A.load()
    rng = np.random.default_rng(3)
    xi = np.ascontiguousarray(rng.normal(size=(3, 6)) * 0.3)
    poses = (A.adop_pose * 3)()
    ref = []
    for k in range(3):
        R, t = _random_pose(rng)
        poses[k] = A.adop_pose((ct.c_float * 9)(*R.reshape(9).tolist()), (ct.c_float * 3)(*t.tolist()))
        T = np.eye(4)
        T[:3, :3], T[:3, 3] = R, t
        ref.append(expm(_hat(xi[k])) @ T)
    assert lib.adop_pose_apply_tangent(xi.ctypes.data_as(ct.c_void_p), poses, 3) == 0
    for k in range(3):
        assert np.max(np.abs(np.array(poses[k].R[:]).reshape(3, 3) - ref[k][:3, :3])) <= 1.2e-7
    bad = xi.copy()
    bad[1, 2] = np.nan
    before = [list(p.R) + list(p.t) for p in poses]
    assert lib.adop_pose_apply_tangent(bad.ctypes.data_as(ct.c_void_p), poses, 3) == 1
    assert [list(p.R) + list(p.t) for p in poses] == before  # nothing changed
    assert lib.adop_pose_apply_tangent(None, None, -1) == 1
    assert lib.adop_pose_apply_tangent(None, None, 0) == 0
