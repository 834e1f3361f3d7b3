"""Helpers of the GPU-vs-oracle parity tests: run the CUDA library and the CPU
oracle on the same seeded inputs and compare with the stated tolerances.

Tolerances (relative, written from the arithmetic of each output):
  keys, counts         bit-exact (integer results of the FP32 projection contract)
  features (FP32 sums) |gpu - ref| <= 1e-5 * max(|ref|, rms(ref)) per element
  BF16 / FP16 image    the same with 2e-2 (one BF16 rounding of the output is 2^-9)
  per-point gradients  |gpu - ref| <= 1e-4 * max(|ref|, rms(ref)) per element
  pose / intrinsics    |gpu - ref| <= 1e-4 * sum over (point, layer) of |term|
  with an environment map, pixels where no point lands hold a bilinear sample
  whose texel coordinates the GPU computes in FP32 (inverse camera, rotation,
  atan2 / acos): a direction error of at most ~4e-6 rad moves them by
  (env_w / 2 pi + env_h / pi) 4e-6 texels, which for the maps used (64 x 128,
  neighbouring texels within ~0.3, values ~0.5) is <= 5e-5 absolute, so the
  image and gradients use 1e-4 there; dL/dE sums FP32 weights w G whose
  weights carry the same coordinate error: 1e-3.
"""
from __future__ import annotations

import numpy as np

RTOL_FEAT_F32 = 1e-5
RTOL_FEAT_LOWP = 2e-2
RTOL_GRAD = 1e-4
RTOL_REDUCED = 1e-4
RTOL_ENV_IMG = 1e-4
RTOL_ENV_GRAD = 1e-3

U64_MAX = np.iinfo(np.uint64).max


def rel_err(gpu, ref):
    """max over elements of |gpu - ref| / max(|ref|, rms(ref))."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(ref * ref)))
    den = np.maximum(np.abs(ref), rms)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(np.abs(gpu - ref) / den))


def assert_close(gpu, ref, rtol, what=""):
    e = rel_err(gpu, ref)
    assert e <= rtol, f"{what}: relative error {e:.3e} > {rtol:.1e}"
    return e


def assert_reduced(gpu, ref, abs_sum, rtol=RTOL_REDUCED, what=""):
    gpu, ref, abs_sum = (np.asarray(v, np.float64) for v in (gpu, ref, abs_sum))
    bound = rtol * np.maximum(abs_sum, 1e-30)
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), f"{what}: gpu {gpu} ref {ref} bound {bound}"


def torch_dtype(name):
    import torch
    return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[name]


def feat_tensor(scene, dtype: str, device="cuda"):
    import torch
    f = scene.feat_as(dtype)
    if dtype == "bf16":
        return torch.from_numpy(f.view(np.int16).copy()).to(device).view(torch.bfloat16)
    return torch.from_numpy(np.ascontiguousarray(f)).to(device)


def to_np(t):
    import torch
    if t.dtype == torch.bfloat16:
        return t.float().cpu().numpy()
    return t.cpu().numpy()


def gpu_run(adop, scene, cams, dtype="f32", levels=4, alpha=0.01, znear=1e-3, background=None, flags=0,
            grads=None, out_dtype="f32", keep_state=True, backward=True, normals=False, crf=True,
            grad_assign=False, init=0.0, vis=True, discard=None, env=None, grad_dtype="f32", grad_feat_dtype="f32"):
    """Forward (+ backward) through the C ABI; returns numpy results.
    grad_dtype / grad_feat_dtype: storage types of the upstream gradients and
    of dL/dtau ("f32", "bf16", "f16")."""
    import torch
    dev = "cuda"
    xyz = torch.from_numpy(scene.xyz).to(dev)
    feat = feat_tensor(scene, dtype, dev)
    nrm = torch.from_numpy(scene.normals).to(dev) if normals else None
    rad = None if discard is None else torch.from_numpy(discard[0]).to(dev)
    bet = None if discard is None else torch.from_numpy(discard[1]).to(dev)
    pts = adop.Points(xyz, feat, nrm, rad, bet)
    bg = None if background is None else torch.tensor(np.asarray(background, np.float32), device=dev)
    if grad_assign:
        flags |= adop.ADOP_FLAG_GRAD_ASSIGN
    # the library's map is texel-major (h x w x c); the oracle's is planar (c x h x w)
    env_t = None if env is None else \
        torch.from_numpy(np.ascontiguousarray(np.moveaxis(np.asarray(env, np.float32), 0, -1))).to(dev)
    params = adop.Params(levels, alpha, znear, bg, flags, 1.5 if discard is None else discard[2], env_t)
    luts = [torch.from_numpy(np.ascontiguousarray(c.crf, np.float32)).to(dev)
            if (crf and getattr(c, "crf", None) is not None) else None for c in cams]
    frames = [adop.Frame.alloc(c, scene.c, levels, torch_dtype(out_dtype), keep_state, dev,
                               scene.n if vis else None) for c in cams]
    ws = adop.alloc_workspace(pts, cams, params, luts, dev)
    adop.adop_render_forward(pts, cams, params, frames, ws, crf_luts=luts)
    out = {"frames": frames}
    if keep_state:
        out["keys"] = [f.key.cpu().numpy().view(np.uint64) for f in frames]
        out["cnt"] = [f.count.cpu().numpy().view(np.uint32) for f in frames]
    out["img"] = [np.concatenate([to_np(im).ravel() for im in f.images]) for f in frames]
    if backward:
        n, c = scene.n, scene.c
        gfeat = torch.full((n, c), init, dtype=torch_dtype(grad_feat_dtype), device=dev)
        gxyz = torch.full((n, 3), init, dtype=torch.float32, device=dev)
        gpose = torch.full((len(cams), 6), init, dtype=torch.float32, device=dev)
        gintr = torch.full((len(cams), 6), init, dtype=torch.float32, device=dev)
        gimgs = [[torch.from_numpy(np.ascontiguousarray(g, np.float32)).to(dev).to(torch_dtype(grad_dtype))
                  for g in gk] for gk in grads]
        adop.adop_render_backward(pts, cams, params, frames, gimgs, gfeat, gxyz, gpose, gintr, ws, crf_luts=luts)
        torch.cuda.synchronize()
        out["dfeat"] = gfeat.float().cpu().numpy().astype(np.float64) - init
        out["dxyz"] = gxyz.cpu().numpy().astype(np.float64) - init
        out["dpose"] = gpose.cpu().numpy().astype(np.float64) - init
        out["dintr"] = gintr.cpu().numpy().astype(np.float64) - init
        if env is not None and keep_state:
            genv = torch.zeros_like(env_t)
            adop.adop_env_backward(cams, params, c, frames, gimgs, genv, crf_luts=luts)
            torch.cuda.synchronize()
            out["denv"] = np.moveaxis(genv.cpu().numpy().astype(np.float64), -1, 0)
    torch.cuda.synchronize()
    return out


def oracle_run(orc, scene, cams, dtype="f32", levels=4, alpha=0.01, znear=1e-3, background=None, grads=None,
               normals=False, epilogue=False, all_projected=False, backward=True, discard=None, leaky=False,
               log_desc=False, env=None, threads=0):
    """The oracle on the same inputs: per camera forward (+ backward), summed
    over cameras for the per-point gradients.  On every core by default: the
    oracle's results do not depend on its thread count (its pose and
    intrinsics sums only in FP64 rounding, far below every tolerance here)."""
    feat = scene.feat_as(dtype)
    res = {"keys": [], "cnt": [], "img": [], "dpose": [], "dintr": [], "dpose_abs": [], "dintr_abs": []}
    dfeat = np.zeros((scene.n, scene.c))
    dxyz = np.zeros((scene.n, 3))
    denv = None if env is None else np.zeros(np.shape(env))
    for k, cam in enumerate(cams):
        kw = {} if discard is None else {"radius": discard[0], "beta": discard[1], "gamma": discard[2]}
        kw["log_desc"] = log_desc
        kw["env"] = None if env is None else np.asarray(env, np.float64)
        f = orc.forward(scene.xyz, feat, cam, levels, alpha, znear, background,
                        scene.normals if normals else None, threads=threads, **kw)
        res["keys"].append(f.keys)
        res["cnt"].append(f.cnt)
        img = f.img.copy()
        G = None if grads is None else np.concatenate([np.asarray(g, np.float64).ravel() for g in grads[k]])
        if epilogue and getattr(cam, "epilogue", False):
            c, h, w = scene.c, cam.h, cam.w
            img0, dgain = orc.epilogue(f.img[:c * h * w].reshape(c, h, w), cam.ev, cam.wb, cam.vig_c, cam.vig_a,
                                       cam.crf, want_grad=True, leaky=leaky)
            img[:c * h * w] = img0.ravel()
            if G is not None:
                G = G.copy()
                G[:c * h * w] *= dgain.ravel()
        res["img"].append(img)
        if backward and G is not None:
            if env is not None:
                denv += orc.env_grad(f, cam, G, denv.shape)
            b = orc.backward(f, scene.xyz, feat, cam, G, alpha, background, all_projected, log_desc,
                             threads=threads, layer_grads=False)
            dfeat += b.dfeat
            dxyz += b.dxyz
            for key in ("dpose", "dintr", "dpose_abs", "dintr_abs"):
                res[key].append(getattr(b, key))
    res["dfeat"], res["dxyz"] = dfeat, dxyz
    if denv is not None:
        res["denv"] = denv
    return res


# |x - boundary| below which the GPU's FP32 and the oracle's FP64 response
# input x may fall on different sides of a response-curve knot or of the ends
# of [0, 1] (x carries the FP32 error of the blended mean, ~1e-6 absolute)
EPI_AMBIGUOUS = 1e-5


def epilogue_decidable_grads(orc, scene, cams, grads, dtype="f32", levels=4, leaky=False, env=None):
    """The upstream gradients with layer 0's channels 0..2 zeroed where the
    photometric response's input x lies within EPI_AMBIGUOUS of a knot of the
    LUT or of 0 or 1.  The response's slope jumps there, so which slope
    chains the gradient is decided by the last bits of x, and both slopes are
    correct answers; zeroing G there (on both sides) compares only what is
    unique.  Uses the oracle's forward for x."""
    out = []
    for k, cam in enumerate(cams):
        G = [np.array(g, np.float64, copy=True) for g in grads[k]]
        crf = getattr(cam, "crf", None)
        if getattr(cam, "epilogue", False) and crf is not None:
            f = orc.forward(scene.xyz, scene.feat_as(dtype), cam, levels,
                            env=None if env is None else np.asarray(env, np.float64))
            c, h, w = scene.c, cam.h, cam.w
            I = f.img[:c * h * w].reshape(c, h, w)
            blended = f.cnt[:h * w].reshape(h, w) > 0  # empty pixels hold the same constant on both sides
            v, u = np.mgrid[0:h, 0:w]
            r2 = (u / w - cam.vig_c[0]) ** 2 + (v / h - cam.vig_c[1]) ** 2
            a = cam.vig_a
            vig = 1.0 + r2 * (a[0] + r2 * (a[1] + r2 * a[2]))
            n1 = np.asarray(crf).shape[-1] - 1
            for ch in range(min(c, 3)):
                x = I[ch] * 2.0 ** -cam.ev * cam.wb[ch] * vig
                t = np.clip(x, 0.0, 1.0) * n1
                near_knot = (np.abs(t - np.round(t)) / n1 < EPI_AMBIGUOUS) & (x > -EPI_AMBIGUOUS) & \
                    (x < 1.0 + EPI_AMBIGUOUS)
                near_end = (np.abs(x) < EPI_AMBIGUOUS) | (np.abs(x - 1.0) < EPI_AMBIGUOUS)
                G[0][ch][(near_knot | near_end) & blended] = 0.0
        out.append(G)
    return out


def compare(gpu, ref, dtype="f32", out_dtype="f32", check_state=True, backward=True, env=False):
    """Assert parity of every output; returns the measured relative errors."""
    errs = {}
    rt_img = RTOL_FEAT_F32 if out_dtype == "f32" else RTOL_FEAT_LOWP
    rt_grad = RTOL_GRAD
    if env:
        rt_img, rt_grad = max(rt_img, RTOL_ENV_IMG), max(RTOL_GRAD, RTOL_ENV_IMG)
    for k in range(len(ref["img"])):
        if check_state:
            assert np.array_equal(gpu["keys"][k], ref["keys"][k]), \
                f"camera {k}: {(gpu['keys'][k] != ref['keys'][k]).sum()} keys differ"
            assert np.array_equal(gpu["cnt"][k], ref["cnt"][k]), f"camera {k}: counts differ"
        errs[f"img{k}"] = assert_close(gpu["img"][k], ref["img"][k], rt_img, f"camera {k} image")
    if backward:
        errs["dfeat"] = assert_close(gpu["dfeat"], ref["dfeat"], rt_grad, "dL/dtau")
        errs["dxyz"] = assert_close(gpu["dxyz"], ref["dxyz"], rt_grad, "dL/dx")
        if "denv" in ref and "denv" in gpu:
            errs["denv"] = assert_close(gpu["denv"], ref["denv"], RTOL_ENV_GRAD, "dL/dE")
        for k in range(len(ref["dpose"])):
            assert_reduced(gpu["dpose"][k], ref["dpose"][k], ref["dpose_abs"][k], what=f"camera {k} dL/dxi")
            assert_reduced(gpu["dintr"][k], ref["dintr"][k], ref["dintr_abs"][k], what=f"camera {k} dL/dK")
    return errs
