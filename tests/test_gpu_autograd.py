"""The torch.autograd.Function over the C ABI: gradients with respect to
descriptors, positions, the tangent-space pose and the intrinsics against the
oracle (whose chain rule is pinned by finite differences), descriptor
gradients against finite differences of the GPU render, and the recompute
policy (no per-pixel state kept) against the kept-state policy."""
import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, RTOL_GRAD, assert_close, assert_reduced

pytestmark = pytest.mark.gpu


def _setup(torch):
    sc = scenes.tiny_spheres(12000, 4, seed=71)
    cams = []
    for k, (w, h) in enumerate([(160, 120), (128, 96)]):
        R, t = scenes.look_at(np.array([np.cos(k + 0.3), 0.2, np.sin(k + 0.3)]) * 2.4 + 0.5, np.full(3, 0.5))
        cams.append(scenes.Camera(w, h, 0.9 * w, 0.9 * w, w / 2, h / 2, k1=0.03, k2=-0.01, R=R, t=t))
    G = [scenes.upstream_grad(c.w, c.h, 4, 4, 80 + k) for k, c in enumerate(cams)]
    return sc, cams, G


def _loss(imgs, Gt):
    return sum((im * g).sum() for row, grow in zip(imgs, Gt) for im, g in zip(row, grow))


@pytest.mark.parametrize("keep_state", [True, False])
def test_autograd_against_oracle(adop, orc, keep_state):
    import torch
    from paper_2110_06635_gb300.autograd import rasterize
    sc, cams, G = _setup(torch)
    xyz = torch.from_numpy(sc.xyz).cuda().requires_grad_()
    feat = torch.from_numpy(sc.feat).cuda().requires_grad_()
    xi = torch.zeros((2, 6), dtype=torch.float32, device="cuda", requires_grad=True)
    intr = torch.tensor([[c.fx, c.fy, c.cx, c.cy, c.k1, c.k2] for c in cams], dtype=torch.float32,
                        requires_grad=True)
    imgs = rasterize(xyz, feat, cams, xi, intr, keep_state=keep_state)
    Gt = [[torch.from_numpy(g).cuda() for g in row] for row in G]
    _loss(imgs, Gt).backward()
    dfeat = np.zeros((sc.n, 4))
    dxyz = np.zeros((sc.n, 3))
    for k, cam in enumerate(cams):
        f = orc.forward(sc.xyz, sc.feat, cam)
        b = orc.backward(f, sc.xyz, sc.feat, cam, np.concatenate([g.ravel() for g in G[k]]).astype(np.float64))
        dfeat += b.dfeat
        dxyz += b.dxyz
        assert_reduced(xi.grad[k].cpu().numpy(), b.dpose, b.dpose_abs, what="dL/dxi")
        assert_reduced(intr.grad[k].numpy(), b.dintr, b.dintr_abs, what="dL/dK")
    assert_close(feat.grad.cpu().numpy(), dfeat, RTOL_GRAD, "dL/dtau")
    assert_close(xyz.grad.cpu().numpy(), dxyz, RTOL_GRAD, "dL/dx")


def test_descriptor_gradient_matches_finite_differences(adop):
    import torch
    from paper_2110_06635_gb300.autograd import rasterize
    sc, cams, G = _setup(torch)
    Gt = [[torch.from_numpy(g).cuda() for g in row] for row in G]
    xyz = torch.from_numpy(sc.xyz).cuda()
    feat = torch.from_numpy(sc.feat).cuda().requires_grad_()
    _loss(rasterize(xyz, feat, cams), Gt).backward()
    g = feat.grad.cpu().numpy()
    rng = np.random.default_rng(3)
    with torch.no_grad():
        base = _loss(rasterize(xyz, feat.detach(), cams), Gt).item()
        for i in rng.choice(np.nonzero(np.abs(g).sum(1))[0], 12, replace=False):
            for ch in range(4):
                f2 = feat.detach().clone()
                f2[i, ch] += 1.0   # the image is linear in the descriptors
                fd = _loss(rasterize(xyz, f2, cams), Gt).item() - base
                assert abs(fd - g[i, ch]) <= 2e-3 * max(1.0, abs(g[i, ch])), (i, ch, fd, g[i, ch])


def test_tangent_pose_is_applied(adop):
    """A non-zero xi renders exp(xi)(R, t): the same image as a camera whose
    pose was multiplied on the host."""
    import torch
    from scipy.linalg import expm
    from paper_2110_06635_gb300.autograd import rasterize
    sc, cams, _ = _setup(torch)
    xyz = torch.from_numpy(sc.xyz).cuda()
    feat = torch.from_numpy(sc.feat).cuda()
    xi = torch.tensor([[0.01, -0.02, 0.03, 0.02, -0.01, 0.015]] * 2, device="cuda")
    a = rasterize(xyz, feat, cams, xi)
    moved = []
    for c in cams:
        T = np.eye(4)
        T[:3, :3], T[:3, 3] = c.R, c.t
        x = xi[0].cpu().numpy().astype(np.float64)
        hat = np.zeros((4, 4))
        hat[:3, :3] = [[0, -x[5], x[4]], [x[5], 0, -x[3]], [-x[4], x[3], 0]]
        hat[:3, 3] = x[:3]
        T = expm(hat) @ T  # the twist's matrix exponential, independent of the library
        moved.append(c.with_pose(T[:3, :3], T[:3, 3]))
    b = rasterize(xyz, feat, moved)
    # same pixels and blends; FP32 sums may differ in atomic summation order only
    for ra, rb in zip(a, b):
        for ia, ib in zip(ra, rb):
            assert_close(ia.cpu().numpy(), ib.cpu().numpy(), RTOL_FEAT_F32, "exp(xi)(R,t) render")


def test_bf16_descriptors_get_bf16_gradients(adop):
    import torch
    from paper_2110_06635_gb300.autograd import rasterize
    sc, cams, G = _setup(torch)
    Gt = [[torch.from_numpy(g).cuda() for g in row] for row in G]
    feat = torch.from_numpy(sc.feat).cuda().to(torch.bfloat16).requires_grad_()
    _loss(rasterize(torch.from_numpy(sc.xyz).cuda(), feat, cams, out_dtype=torch.bfloat16), Gt).backward()
    assert feat.grad.dtype == torch.bfloat16 and torch.isfinite(feat.grad.float()).all()
