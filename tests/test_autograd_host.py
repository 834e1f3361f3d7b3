"""Host-side parts of the autograd wrapper: the SE(3) exponential used to
apply the tangent-space pose increment (Eq. tangent) against scipy's matrix
exponential of the twist."""
import numpy as np
from scipy.linalg import expm


def _hat(xi):
    nu, om = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]]
    M[:3, 3] = nu
    return M


def test_se3_exp_matches_matrix_exponential():
    from paper_2110_06635_gb300.autograd import se3_exp
    rng = np.random.default_rng(0)
    for scale in (1e-10, 1e-4, 0.1, 1.0, 2.5):
        for _ in range(20):
            xi = rng.normal(size=6) * scale
            assert np.allclose(se3_exp(xi), expm(_hat(xi)), rtol=0, atol=1e-12)
