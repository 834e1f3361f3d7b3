"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.  Keys and counts bit-exact; features and gradients
within the tolerances stated in tests/parity.py."""
import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, RTOL_GRAD, assert_close, compare, epilogue_decidable_grads, gpu_run, oracle_run, torch_dtype

pytestmark = pytest.mark.gpu


def _grads(cams, c, levels, seed):
    return [scenes.upstream_grad(cam.w, cam.h, levels, c, seed + k) for k, cam in enumerate(cams)]


@pytest.fixture(scope="module")
def tiny():
    return scenes.config(1)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_tiny_config_fwd_bwd(adop, orc, tiny, dtype):
    """20,000 points on 3 spheres, 256^2, C = 4, L = 4, alpha = 0.01."""
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 7)
    g = gpu_run(adop, sc, cams, dtype, grads=G)
    r = oracle_run(orc, sc, cams, dtype, grads=G)
    compare(g, r, dtype)


@pytest.mark.parametrize("c", [1, 2, 3, 4, 8, 16])
def test_channel_counts_ragged_image(adop, orc, c):
    """Every compiled channel count on an odd-sized image (ragged layers and
    tails) with a point count that is not a multiple of the block size."""
    sc = scenes.tiny_spheres(4099, c, seed=31)
    cam = scenes.Camera(193, 97, 160.0, 160.0, 96.3, 48.7, k1=0.02, k2=-0.01, p1=0.001, p2=-0.002,
                        R=np.eye(3, dtype=np.float32), t=np.array([-0.4, -0.4, 2.2], np.float32))
    G = _grads([cam], c, 4, 11)
    bg = np.linspace(-0.5, 0.5, c)
    g = gpu_run(adop, sc, [cam], "f32", background=bg, grads=G)
    r = oracle_run(orc, sc, [cam], "f32", background=bg, grads=G)
    compare(g, r)


@pytest.mark.parametrize("out_dtype", ["bf16", "f16"])
def test_low_precision_output(adop, orc, tiny, out_dtype):
    sc, cams = tiny
    g = gpu_run(adop, sc, cams, "bf16", out_dtype=out_dtype, backward=False)
    r = oracle_run(orc, sc, cams, "bf16", backward=False)
    compare(g, r, "bf16", out_dtype, backward=False)


def test_recompute_matches_kept_state(adop, orc, tiny):
    """Frames without key/count/acc: the backward re-renders (Sec. 3.1,
    implementation details) and must give the kept-state results."""
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 7)
    g = gpu_run(adop, sc, cams, "f32", grads=G, keep_state=False)
    r = oracle_run(orc, sc, cams, "f32", grads=G)
    compare(g, r, check_state=False)


def test_without_visibility_mask(adop, orc, tiny):
    """Kept state without the per-point layer mask: the backward takes the
    fuzzy decision from the pixel records instead, with the same results."""
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 7)
    for flags in (0, adop.ADOP_FLAG_GRAD_ALL_PROJECTED):
        g = gpu_run(adop, sc, cams, "f32", grads=G, vis=False, flags=flags)
        r = oracle_run(orc, sc, cams, "f32", grads=G, all_projected=bool(flags))
        compare(g, r)


def test_accumulate_and_assign(adop, orc, tiny):
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 7)
    r = oracle_run(orc, sc, cams, "f32", grads=G)
    g = gpu_run(adop, sc, cams, "f32", grads=G, init=1.0)
    compare(g, r)
    g = gpu_run(adop, sc, cams, "f32", grads=G, grad_assign=True)
    compare(g, r)


def test_multi_camera(adop, orc):
    """Three views of one cloud in one call: per-point gradients sum over views."""
    sc = scenes.tiny_spheres(6000, 4, seed=41)
    cams = []
    for k, (w, h) in enumerate([(160, 120), (131, 77), (96, 96)]):
        R, t = scenes.look_at(np.array([np.cos(k), 0.3, np.sin(k)]) * 2.5 + 0.5, np.full(3, 0.5))
        cams.append(scenes.Camera(w, h, 0.9 * w, 0.9 * w, w / 2, h / 2, k1=0.01, R=R, t=t))
    G = _grads(cams, sc.c, 4, 17)
    for assign in (False, True):
        g = gpu_run(adop, sc, cams, "f32", grads=G, grad_assign=assign)
        r = oracle_run(orc, sc, cams, "f32", grads=G)
        compare(g, r)


def test_all_projected_flag(adop, orc, tiny):
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 9)
    g = gpu_run(adop, sc, cams, "f32", grads=G, flags=adop.ADOP_FLAG_GRAD_ALL_PROJECTED)
    r = oracle_run(orc, sc, cams, "f32", grads=G, all_projected=True)
    compare(g, r)


def test_normal_culling(adop, orc, tiny):
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 5)
    g = gpu_run(adop, sc, cams, "f32", grads=G, normals=True, flags=adop.ADOP_FLAG_NORMAL_CULL)
    r = oracle_run(orc, sc, cams, "f32", grads=G, normals=True)
    compare(g, r)


def test_photometric_epilogue(adop, orc):
    """Exposure, white balance, vignette and response curve on layer 0 (Sec. 3.3),
    forward and chained into the backward."""
    sc = scenes.tiny_spheres(8000, 4, seed=51)
    cams = scenes.orbit_cameras(2, seed=52, radius=2.5, resolutions=((128, 96), (100, 75)))
    for cam in cams:
        R, t = scenes.look_at(-cam.R.T @ cam.t, np.full(3, 0.5))
        cam.R, cam.t = R, t
    sc.feat = np.abs(sc.feat) * 0.5  # radiance-like descriptors
    G = epilogue_decidable_grads(orc, sc, cams, _grads(cams, sc.c, 4, 53))
    g = gpu_run(adop, sc, cams, "f32", grads=G, flags=adop.ADOP_FLAG_EPILOGUE)
    r = oracle_run(orc, sc, cams, "f32", grads=G, epilogue=True)
    compare(g, r)


def test_empty_and_degenerate_inputs(adop, orc):
    cam = scenes.tiny_camera()
    bg = np.array([0.1, 0.2, 0.3, 0.4])
    # no points at all: background everywhere, gradients untouched
    empty = scenes.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32))
    G = _grads([cam], 4, 4, 3)
    g = gpu_run(adop, empty, [cam], "f32", background=bg, grads=G)
    r = oracle_run(orc, empty, [cam], "f32", background=bg, grads=G)
    compare(g, r)
    # every point behind the camera (z <= znear) or outside the image
    sc = scenes.tiny_spheres(3000, 4, seed=61)
    behind = scenes.Camera(256, 256, 205.0, 205.0, 128.0, 128.0, R=np.eye(3, dtype=np.float32),
                           t=np.array([0, 0, -5], np.float32))
    g = gpu_run(adop, sc, [behind], "f32", background=bg, grads=G)
    r = oracle_run(orc, sc, [behind], "f32", background=bg, grads=G)
    compare(g, r)
    assert np.all(g["cnt"][0] == 0)


def test_exact_half_pixel_ties(adop, orc):
    """Projections exactly on .5 pixel boundaries round half to even on both sides."""
    w, h = 16, 8
    cam = scenes.Camera(w, h, 1.0, 1.0, 0.0, 0.0, R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32))
    u = np.array([0.5, 1.5, 2.5, 3.5, 4.5, 7.5, 8.0, 15.5, 14.5, 6.5], np.float32)
    v = np.array([0.5, 1.5, 2.5, 3.5, 4.5, 6.5, 7.5, 0.0, 2.0, 5.5], np.float32)
    z = np.full(10, 2.0, np.float32)
    xyz = np.stack([u * z, v * z, z], 1).astype(np.float32)
    sc = scenes.Scene(xyz, np.arange(20, dtype=np.float32).reshape(10, 2), np.zeros((10, 3), np.float32))
    G = _grads([cam], 2, 3, 4)
    g = gpu_run(adop, sc, [cam], "f32", levels=3, grads=G)
    r = oracle_run(orc, sc, [cam], "f32", levels=3, grads=G)
    compare(g, r)


def test_alpha_zero_and_large_alpha(adop, orc, tiny):
    sc, cams = tiny
    G = _grads(cams, sc.c, 4, 8)
    for alpha in (0.0, 0.2):
        g = gpu_run(adop, sc, cams, "f32", alpha=alpha, grads=G)
        r = oracle_run(orc, sc, cams, "f32", alpha=alpha, grads=G)
        compare(g, r)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_log_descriptors(adop, orc, tiny, dtype):
    """Logarithmic descriptors (Sec. 3.2): exp(tau) is blended; dL/dtau of the stored values."""
    sc, cams = tiny
    sc = scenes.Scene(sc.xyz, (sc.feat * 0.5).astype(np.float32), sc.normals)
    G = _grads(cams, sc.c, 4, 13)
    for vis in (True, False):
        g = gpu_run(adop, sc, cams, dtype, grads=G, flags=adop.ADOP_FLAG_LOG_DESCRIPTORS, vis=vis)
        r = oracle_run(orc, sc, cams, dtype, grads=G, log_desc=True)
        compare(g, r, dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_fisheye_camera(adop, orc, dtype):
    """The fisheye model (stereographic, distance as depth) close to the
    spheres, with points far off axis and some behind the image plane."""
    from scipy.spatial.transform import Rotation
    sc = scenes.tiny_spheres(12000, 4, seed=81)
    R = Rotation.from_rotvec([0.05, -0.1, 0.02]).as_matrix().astype(np.float32)
    cam = scenes.Camera(160, 120, 48.0, 48.0, 80.5, 60.5, k1=0.05, k2=-0.02, k3=0.004, R=R,
                        t=np.array([-0.45, -0.35, 0.6], np.float32), model=1)
    G = _grads([cam], 4, 4, 21)
    g = gpu_run(adop, sc, [cam], dtype, grads=G)
    r = oracle_run(orc, sc, [cam], dtype, grads=G)
    compare(g, r, dtype)
    assert (g["cnt"][0] > 0).sum() > 1000


@pytest.mark.parametrize("gdt", ["bf16", "f16"])
def test_16bit_gradient_io(adop, orc, gdt):
    """Upstream gradients stored in BF16 / FP16 and dL/dtau returned in the same
    type (assigned, one camera).  The gradients are rounded to that type once
    on the host, so the GPU and the oracle see the same values: dL/dx, pose and
    intrinsics within the FP32 tolerances, dL/dtau within one 16-bit rounding
    of the output (RTOL_FEAT_LOWP)."""
    import torch
    from parity import RTOL_FEAT_LOWP, assert_reduced
    sc = scenes.tiny_spheres(20000, 8, seed=71)
    cams = [scenes.tiny_camera()]
    G = [[torch.from_numpy(g).to(torch_dtype(gdt)).float().numpy()
          for g in scenes.upstream_grad(c.w, c.h, 4, sc.c, 72)] for c in cams]
    g = gpu_run(adop, sc, cams, "bf16", grads=G, grad_assign=True, grad_dtype=gdt, grad_feat_dtype=gdt)
    r = oracle_run(orc, sc, cams, "bf16", grads=G)
    assert np.array_equal(g["keys"][0], r["keys"][0]) and np.array_equal(g["cnt"][0], r["cnt"][0])
    assert_close(g["dfeat"], r["dfeat"], RTOL_FEAT_LOWP, f"dL/dtau stored as {gdt}")
    assert_close(g["dxyz"], r["dxyz"], RTOL_GRAD, "dL/dx")
    assert_reduced(g["dpose"][0], r["dpose"][0], r["dpose_abs"][0], what="dL/dxi")
    assert_reduced(g["dintr"][0], r["dintr"][0], r["dintr_abs"][0], what="dL/dK")
    assert np.abs(r["dfeat"]).max() > 0 and np.abs(r["dxyz"]).max() > 0


def test_layer_mask_buffer_only_4_byte_aligned(adop, orc):
    """The ABI asks only 4-byte alignment of a caller's layer-mask buffer: a
    buffer 4 bytes past an aligned start (and a point count that is not a
    multiple of 4) gives the oracle's results."""
    import torch
    from parity import assert_reduced
    sc = scenes.tiny_spheres(20003, 8, seed=75)  # n not a multiple of 4
    cams = [scenes.tiny_camera()]
    G = [scenes.upstream_grad(c.w, c.h, 4, sc.c, 76) for c in cams]
    r = oracle_run(orc, sc, cams, "f32", grads=G)
    dev = "cuda"
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(4, 0.01, 1e-3, None, adop.ADOP_FLAG_GRAD_ASSIGN)
    fr = adop.Frame.alloc(cams[0], sc.c, 4, torch.float32, True, dev, sc.n)
    fr.vis = torch.empty(sc.n + 1, dtype=torch.int32, device=dev)[1:]  # 4 bytes past an aligned start
    assert fr.vis.data_ptr() % 16 == 4
    ws = adop.alloc_workspace(pts, cams, params, None, dev)
    adop.adop_render_forward(pts, cams, params, [fr], ws)
    out = [torch.empty((sc.n, sc.c), device=dev), torch.empty((sc.n, 3), device=dev),
           torch.zeros((1, 6), device=dev), torch.zeros((1, 6), device=dev)]
    adop.adop_render_backward(pts, cams, params, [fr], [[torch.from_numpy(x).to(dev) for x in G[0]]], *out, ws)
    assert np.array_equal(fr.key.cpu().numpy().view(np.uint64), r["keys"][0])
    assert_close(out[0].cpu().numpy(), r["dfeat"], RTOL_GRAD, "dL/dtau")
    assert_close(out[1].cpu().numpy(), r["dxyz"], RTOL_GRAD, "dL/dx")
    assert_reduced(out[2].cpu().numpy()[0], r["dpose"][0], r["dpose_abs"][0], what="dL/dxi")
    assert_reduced(out[3].cpu().numpy()[0], r["dintr"][0], r["dintr_abs"][0], what="dL/dK")


def test_layer_masks_match_the_oracle(adop, orc):
    """The forward's per-point layer mask (include/adop.h, adop_frame.vis,
    bits 0-7) equals the oracle's fuzzy-test membership bit for bit: the
    point passes z <= f32(z_min (1 + alpha)) at its layer-l pixel, with z_min
    from the oracle's keys; a point count that is not a multiple of 32."""
    import torch
    sc = scenes.tiny_spheres(20003, 8, seed=81)
    cam = scenes.tiny_camera()
    f = orc.forward(sc.xyz, sc.feat, cam, 4, 0.01, 1e-3)
    keys = [k.reshape(-1) for k in f.layer_keys()]
    a1 = np.float32(1.01)
    mask = np.zeros(sc.n, np.uint32)
    for l in range(4):
        p = f.pix[:, l]
        ok = p >= 0
        zmin = (keys[l][np.where(ok, p, 0)] >> np.uint64(32)).astype(np.uint32).view(np.float32)
        inl = ok & (f.z <= np.float32(zmin * a1))  # FP32 product, rounded once
        mask |= inl.astype(np.uint32) << np.uint32(l)
    assert (mask == 0).any() and (mask != 0).any() and (mask > 1).any()
    dev = "cuda"
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(4, 0.01, 1e-3, None, 0)
    fr = adop.Frame.alloc(cam, sc.c, 4, torch.float32, True, dev, sc.n)
    ws = adop.alloc_workspace(pts, [cam], params, None, dev)
    adop.adop_render_forward(pts, [cam], params, [fr], ws)
    vis = fr.vis.cpu().numpy().view(np.uint32)
    assert np.array_equal(vis & 0xFF, mask)
    assert np.all((vis >> 8)[mask == 0] == 0)  # no tile for a point in no Lambda

def test_sum_buffer_only_16_byte_aligned(adop, orc):
    """The ABI asks 16-byte alignment of a frame's per-pixel sums: with C = 8
    the clear pass uses 256-bit stores only where the sums are 32-byte aligned;
    a buffer 16 bytes past a 32-byte boundary gives the oracle's keys, counts
    and images, the same as an aligned one."""
    import torch
    sc = scenes.tiny_spheres(20000, 8, seed=79)
    cams = [scenes.tiny_camera()]
    r = oracle_run(orc, sc, cams, "f32")
    dev = "cuda"
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(4, 0.01, 1e-3, None, 0)
    for offset in (0, 4):  # floats past a 256-byte aligned start
        fr = adop.Frame.alloc(cams[0], sc.c, 4, torch.float32, True, dev)
        px = fr.key.numel()
        fr.acc = torch.full((px * sc.c + 8,), float("nan"), device=dev)[offset:offset + px * sc.c]
        assert fr.acc.data_ptr() % 32 == 4 * offset
        ws = adop.alloc_workspace(pts, cams, params, None, dev)
        for _ in range(2):  # the second forward clears what the first accumulated
            adop.adop_render_forward(pts, cams, params, [fr], ws)
        assert np.array_equal(fr.key.cpu().numpy().view(np.uint64), r["keys"][0])
        assert np.array_equal(fr.count.cpu().numpy().view(np.uint32), r["cnt"][0])
        img = np.concatenate([im.cpu().numpy().ravel() for im in fr.images])
        assert_close(img, r["img"][0], RTOL_FEAT_F32, "images")


@pytest.mark.gpu
def test_position_gradient_buffer_only_4_byte_aligned(adop, orc):
    """The ABI asks only 4-byte alignment of dL/dx: a buffer 4 bytes past a
    16-byte boundary and one on it give the oracle's results, the zero
    gradients of the points in no Lambda included (filled with NaN before the
    call, so that a point left unwritten shows; a point count that is not a
    multiple of 32, so that the last warp's points are partly out of range)."""
    import torch
    from parity import assert_reduced
    sc = scenes.tiny_spheres(20011, 8, seed=77)
    cams = [scenes.tiny_camera()]
    G = [scenes.upstream_grad(c.w, c.h, 4, sc.c, 78) for c in cams]
    r = oracle_run(orc, sc, cams, "f32", grads=G)
    assert np.sum(~np.any(r["dfeat"] != 0, axis=1)) > 64  # points in no Lambda, whole chunks of them included
    dev = "cuda"
    pts = adop.Points(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.feat).to(dev))
    params = adop.Params(4, 0.01, 1e-3, None, adop.ADOP_FLAG_GRAD_ASSIGN)
    for offset in (0, 1):  # floats past a 256-byte aligned start: 16-byte and 4-byte aligned
        fr = adop.Frame.alloc(cams[0], sc.c, 4, torch.float32, True, dev, sc.n)
        ws = adop.alloc_workspace(pts, cams, params, None, dev)
        adop.adop_render_forward(pts, cams, params, [fr], ws)
        gx = torch.full((sc.n * 3 + 4,), float("nan"), device=dev)[offset:offset + sc.n * 3].view(sc.n, 3)
        assert gx.data_ptr() % 16 == 4 * offset
        out = [torch.full((sc.n, sc.c), float("nan"), device=dev), gx,
               torch.zeros((1, 6), device=dev), torch.zeros((1, 6), device=dev)]
        adop.adop_render_backward(pts, cams, params, [fr], [[torch.from_numpy(x).to(dev) for x in G[0]]], *out,
                                  ws)
        assert_close(out[0].cpu().numpy(), r["dfeat"], RTOL_GRAD, "dL/dtau")
        assert_close(out[1].cpu().numpy(), r["dxyz"], RTOL_GRAD, "dL/dx")
        assert_reduced(out[2].cpu().numpy()[0], r["dpose"][0], r["dpose_abs"][0], what="dL/dxi")
