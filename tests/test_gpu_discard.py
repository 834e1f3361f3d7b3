"""Stochastic point discarding on the GPU (Sec. 3.1, Eq. discard): the world
radius preprocess (4th-nearest point) against the oracle's exhaustive FP64
search, and forward + backward with discarding against the oracle (keys and
counts bit-exact, features and gradients within tolerance)."""
import numpy as np
import pytest

import scenes
from parity import compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def test_point_radius_matches_exhaustive_search(adop, orc):
    import torch
    sc = scenes.tiny_spheres(6000, 1, seed=12)
    xyz = sc.xyz.copy()
    xyz[100:104] = xyz[99]          # five copies: each has 4 neighbours at distance 0
    xyz[5000] = [40.0, -30.0, 25.0]  # an isolated outlier far from the cloud
    want = orc.knn_radius(xyz, 4)
    got = adop.adop_point_radius(torch.from_numpy(xyz).cuda(), 4).cpu().numpy().astype(np.float64)
    inner = np.ones(len(xyz), bool)
    inner[5000] = False
    assert np.allclose(got[inner], want[inner], rtol=1e-5, atol=1e-6)
    assert got[5000] >= want[5000] * (1 - 1e-5)      # the outlier: an upper bound at worst
    assert np.all(got[99:104] == 0.0) and np.all(want[99:104] == 0.0)
    for k in (1, 2, 8):
        w = orc.knn_radius(xyz[:2000], k)
        g = adop.adop_point_radius(torch.from_numpy(xyz[:2000]).cuda(), k).cpu().numpy()
        assert np.allclose(g, w, rtol=1e-5, atol=1e-6), k
    tiny = adop.adop_point_radius(torch.from_numpy(xyz[:4]).cuda(), 4).cpu().numpy()
    assert np.all(np.isinf(tiny))


@pytest.mark.parametrize("keep_state", [True, False])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_discard_fwd_bwd_parity(adop, orc, keep_state, dtype):
    import torch
    sc, cams = scenes.config(1)
    r = orc.knn_radius(sc.xyz, 4).astype(np.float32)
    beta = np.random.default_rng(5).random(sc.n).astype(np.float32)
    G = [scenes.upstream_grad(c.w, c.h, 4, sc.c, 40) for c in cams]
    g = gpu_run(adop, sc, cams, dtype, grads=G, keep_state=keep_state, flags=adop.ADOP_FLAG_DISCARD,
                discard=(r, beta, 1.5))
    ref = oracle_run(orc, sc, cams, dtype, grads=G, discard=(r, beta, 1.5))
    compare(g, ref, dtype, check_state=keep_state)
    # discarding removes points: fewer blends than without
    f0 = orc.forward(sc.xyz, sc.feat_as(dtype), cams[0])
    assert ref["cnt"][0].sum() < f0.cnt.sum()
