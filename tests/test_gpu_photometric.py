"""The photometric camera model on the GPU (Sec. 3.3): parameter gradients
(EV, white balance, vignette, response LUT) against the oracle, the leaky
training response (Eq. resonseleak) forward and chained into the backward,
and a synthetic pose recovery through the tangent-space pose gradient
(Eq. tangent)."""
import numpy as np
import pytest

import scenes
from parity import RTOL_GRAD, assert_close, assert_reduced, compare, epilogue_decidable_grads, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _cams():
    cams = scenes.orbit_cameras(2, seed=52, radius=2.5, resolutions=((128, 96), (100, 75)))
    for cam in cams:
        R, t = scenes.look_at(-cam.R.T @ cam.t, np.full(3, 0.5))
        cam.R, cam.t = R, t
    return cams


def _scene():
    sc = scenes.tiny_spheres(8000, 4, seed=51)
    sc.feat = np.abs(sc.feat) * 0.6  # radiance-like: x covers [0, 1] and beyond
    return sc


@pytest.mark.parametrize("leaky", [False, True])
def test_leaky_epilogue_fwd_bwd(adop, orc, leaky):
    sc, cams = _scene(), _cams()
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 60 + k) for k, c in enumerate(cams)]
    G = epilogue_decidable_grads(orc, sc, cams, G, leaky=leaky)
    flags = adop.ADOP_FLAG_EPILOGUE | (adop.ADOP_FLAG_LEAKY_CRF if leaky else 0)
    g = gpu_run(adop, sc, cams, "f32", grads=G, flags=flags)
    r = oracle_run(orc, sc, cams, "f32", grads=G, epilogue=True, leaky=leaky)
    compare(g, r)


@pytest.mark.parametrize("leaky", [False, True])
def test_photometric_parameter_gradients(adop, orc, leaky):
    import torch
    sc, cams = _scene(), _cams()
    dev = "cuda"
    flags = adop.ADOP_FLAG_EPILOGUE | (adop.ADOP_FLAG_LEAKY_CRF if leaky else 0)
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(4, 0.01, 1e-3, None, flags)
    luts = [torch.from_numpy(np.ascontiguousarray(c.crf, np.float32)).to(dev) for c in cams]
    frames = [adop.Frame.alloc(c, 4, 4, torch.float32, True, dev) for c in cams]
    ws = adop.alloc_workspace(pts, cams, params, luts, dev)
    adop.adop_render_forward(pts, cams, params, frames, ws, crf_luts=luts)
    G0 = [np.random.default_rng(70 + k).normal(size=(4, c.h, c.w)).astype(np.float32) for k, c in enumerate(cams)]
    gp = torch.zeros((2, 9), device=dev)
    n = cams[0].crf.shape[1]
    gcrf = torch.zeros(2 * 3 * n, device=dev)
    adop.adop_photometric_backward(cams, params, 4, frames, [torch.from_numpy(g).to(dev) for g in G0], gp, gcrf,
                                   crf_luts=luts)
    torch.cuda.synchronize()
    gp, gcrf = gp.cpu().numpy(), gcrf.cpu().numpy().reshape(2, 3, n)
    for k, cam in enumerate(cams):
        f = orc.forward(sc.xyz, sc.feat, cam)
        img0 = f.layer_img()[0]
        ref, ref_crf, ref_abs = orc.photometric_grad(img0, G0[k], cam.ev, cam.wb, cam.vig_c, cam.vig_a, cam.crf,
                                                     leaky=leaky, with_abs=True)
        assert_reduced(gp[k], ref, ref_abs, what=f"camera {k} photometric")
        assert_close(gcrf[k], ref_crf, RTOL_GRAD, f"camera {k} response LUT")


def test_pose_recovery_through_the_tangent(adop):
    """Render targets from a true pose, start from a perturbed one and take
    Adam steps on the tangent xi (applied and reset each step, as in the
    paper); the one-pixel spatial gradient must pull the pose back."""
    import torch
    from paper_2110_06635_gb300.autograd import apply_tangent, rasterize
    sc = scenes.tiny_spheres(40000, 4, seed=77)
    p = sc.xyz.astype(np.float64)
    sc.feat = np.stack([np.sin(4 * p[:, 0]), np.cos(4 * p[:, 1]), np.sin(4 * p[:, 2] + 1), np.cos(3 * p[:, 0] + 2 * p[:, 1])],
                       1).astype(np.float32)
    xyz = torch.from_numpy(sc.xyz).cuda()
    feat = torch.from_numpy(sc.feat).cuda()
    R, t = scenes.look_at(np.array([0.4, 0.2, -2.0]), np.full(3, 0.5))
    true = scenes.Camera(160, 120, 150.0, 150.0, 80.0, 60.0, k1=0.01, R=R, t=t)
    with torch.no_grad():
        target = rasterize(xyz, feat, [true])[0]
    xi0 = np.array([0.012, -0.008, 0.01, 0.006, -0.008, 0.004])
    cam = apply_tangent(true, xi0)

    def err(c):
        # mean reprojection distance (layer-0 pixels) of the cloud between the
        # two poses: what image alignment can observe (a lateral translation
        # and a rotation about the orthogonal axis look nearly alike)
        def uv(cc):
            X = p @ np.asarray(cc.R, np.float64).T + np.asarray(cc.t, np.float64)
            return np.stack([cc.fx * X[:, 0] / X[:, 2], cc.fy * X[:, 1] / X[:, 2]], 1)
        return float(np.mean(np.linalg.norm(uv(c) - uv(true), axis=1)))

    e0 = err(cam)
    m = np.zeros(6); v = np.zeros(6)
    lr = 4e-3
    for it in range(150):
        xi = torch.zeros((1, 6), device="cuda", requires_grad=True)
        imgs = rasterize(xyz, feat, [cam], xi)[0]
        loss = sum(((a - b) ** 2).sum() / a.numel() for a, b in zip(imgs, target))
        loss.backward()
        g = xi.grad[0].cpu().numpy().astype(np.float64)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        step = -lr * (m / (1 - 0.9 ** (it + 1))) / (np.sqrt(v / (1 - 0.999 ** (it + 1))) + 1e-12)
        cam = apply_tangent(cam, step)
        lr *= 0.98
    e1 = err(cam)
    assert e1 < 0.3 * e0, (e0, e1)
