"""``torch.autograd.Function`` around the C ABI (Sec. 3.1 forward + backward).

``rasterize(xyz, feat, cameras, xi=None, intrinsics=None, ...)`` renders every
camera's image pyramid and makes it differentiable with respect to

* ``xyz`` (n x 3) -- through the approximate one-pixel spatial gradient,
* ``feat`` (n x c, float32 / bfloat16 / float16 storage; its gradient is FP32
  and is returned in the storage dtype, as autograd requires),
* ``xi`` (n_cam x 6 tangent-space pose increments, (nu, omega)): the pose
  used is exp(xi) (R, t) (Eq. tangent).  As in the paper the optimiser
  updates xi, the caller applies it to the pose and resets it to zero; the
  gradient is that of the left increment at exp(xi) (R, t), which equals
  dL/dxi exactly at xi = 0,
* ``intrinsics`` (n_cam x 6: fx, fy, cx, cy, k1, k2), replacing the cameras'
  values,
* ``env`` (env_h x env_w x c float32, texel-major: the environment map that
  pixels where no point lands show, Sec. 3.1); its gradient needs
  ``keep_state=True``.

``keep_state=True`` keeps each camera's per-pixel key/count/sum buffers and
per-point layer mask for the backward pass; ``keep_state=False`` keeps only
the inputs and the backward pass re-renders the depth and accumulate passes
(the paper's choice: Lambda is never stored).

All arithmetic runs in the library; this module only allocates tensors and
marshals pointers.  The pose exponential (6 numbers per camera) is the
library's host-side adop_pose_apply_tangent, in FP64.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np
import torch

from . import _abi as A


def apply_tangent(cam, xi):
    """The camera with its pose replaced by exp(xi) (R, t) (Eq. tangent): the
    update applied after an optimiser step on the tangent, which is then
    reset to zero.  The exponential and the composition run in the library
    (adop_pose_apply_tangent)."""
    c = copy.copy(cam)
    c.R, c.t = A.adop_pose_apply_tangent(xi, cam.R, cam.t)
    return c


def _effective_cameras(cameras, xi, intrinsics):
    cams = []
    xi_h = None if xi is None else xi.detach().to("cpu", torch.float64).numpy()
    k_h = None if intrinsics is None else intrinsics.detach().to("cpu", torch.float64).numpy()
    for k, cam in enumerate(cameras):
        c = apply_tangent(cam, xi_h[k]) if xi_h is not None and np.any(xi_h[k] != 0) else copy.copy(cam)
        if k_h is not None:
            c.fx, c.fy, c.cx, c.cy, c.k1, c.k2 = (float(v) for v in k_h[k])
        cams.append(c)
    return cams


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, feat, xi, intr, env, cams, params, out_dtype, keep_state, crf_luts, discard, buffers):
        levels = params.levels
        pts = A.Points(xyz.contiguous(), feat.contiguous(), None, *discard)
        frames, ws = buffers  # allocated before the pose was read (see rasterize)
        A.adop_render_forward(pts, cams, params, frames, ws, crf_luts=crf_luts)
        ctx.save_for_backward(xyz, feat)
        # the backward needs the frames' per-pixel state, not their images: the
        # images are this Function's outputs, and holding them here would make
        # a reference cycle (output -> grad_fn -> ctx -> output) that keeps
        # every step's frames and workspace alive until Python's cycle
        # collector runs
        ctx.frames = [dataclasses.replace(f, images=[]) for f in frames]
        ctx.cams, ctx.params, ctx.ws, ctx.crf_luts = cams, params, ws, crf_luts
        ctx.discard = discard
        ctx.has_xi, ctx.has_intr = xi is not None, intr is not None
        ctx.xi_dev = None if xi is None else xi.device
        ctx.intr_dev = None if intr is None else intr.device
        return tuple(im for f in frames for im in f.images)

    @staticmethod
    def backward(ctx, *grad_out):
        xyz, feat = ctx.saved_tensors
        dev = xyz.device
        levels = ctx.params.levels
        ncam = len(ctx.cams)
        # the upstream gradients in their own storage type when they share one
        # the library reads (it widens them to FP32), else as FP32
        given = [g for g in grad_out[:ncam * levels] if g is not None]
        keep = bool(given) and all(g.dtype == given[0].dtype for g in given) and \
            given[0].dtype in (torch.float32, torch.bfloat16, torch.float16)
        gimgs = []
        for k in range(ncam):
            row = []
            for l in range(levels):
                g = grad_out[k * levels + l]
                row.append(None if g is None else (g if keep else g.to(torch.float32)).contiguous())
            gimgs.append(row)
        n, c = feat.shape
        need_xyz = ctx.needs_input_grad[0]
        need_feat = ctx.needs_input_grad[1]
        need_pose = ctx.needs_input_grad[2] or ctx.needs_input_grad[3]
        # dL/dtau is summed in FP32; with one camera the library rounds it to the
        # descriptors' storage type itself, else it is converted afterwards
        gf_dtype = feat.dtype if ncam == 1 else torch.float32
        gfeat = torch.empty((n, c), dtype=gf_dtype, device=dev) if need_feat else None
        gxyz = torch.empty((n, 3), dtype=torch.float32, device=dev) if need_xyz else None
        gpose = torch.zeros((ncam, 6), dtype=torch.float32, device=dev) if need_pose else None
        gintr = torch.zeros((ncam, 6), dtype=torch.float32, device=dev) if need_pose else None
        params = A.Params(ctx.params.levels, ctx.params.alpha, ctx.params.znear, ctx.params.background,
                          ctx.params.flags | A.ADOP_FLAG_GRAD_ASSIGN, ctx.params.gamma, ctx.params.env)
        pts = A.Points(xyz.contiguous(), feat.contiguous(), None, *ctx.discard)
        A.adop_render_backward(pts, ctx.cams, params, ctx.frames, gimgs, gfeat, gxyz, gpose, gintr, ctx.ws,
                               crf_luts=ctx.crf_luts)
        g_env = None
        if ctx.needs_input_grad[4]:
            g_env = torch.zeros_like(ctx.params.env, dtype=torch.float32)
            g32 = [[None if g is None else g.to(torch.float32) for g in row] for row in gimgs]
            A.adop_env_backward(ctx.cams, params, c, ctx.frames, g32, g_env, crf_luts=ctx.crf_luts)
        g_feat = None if gfeat is None else gfeat.to(feat.dtype)
        g_xi = None if not ctx.needs_input_grad[2] else gpose.to(ctx.xi_dev)
        g_intr = None if not ctx.needs_input_grad[3] else gintr.to(ctx.intr_dev)
        return gxyz, g_feat, g_xi, g_intr, g_env, None, None, None, None, None, None, None


def rasterize(xyz, feat, cameras, xi=None, intrinsics=None, levels=4, alpha=0.01, znear=1e-3, background=None,
              flags=0, out_dtype=torch.float32, keep_state=True, crf_luts=None, radius=None, beta=None, gamma=1.5,
              env=None):
    """Differentiable render of every camera; returns [camera][layer] images
    (c x h_l x w_l).  See the module docstring for the gradients.  With
    radius and beta (float32 per point), stochastic point discarding
    (Eq. discard) with threshold gamma; with env (env_h x env_w x c float32),
    empty pixels sample the environment map."""
    if radius is not None:
        flags |= A.ADOP_FLAG_DISCARD
    if env is not None and env.requires_grad and not keep_state:
        raise ValueError("the environment map's gradient needs keep_state=True (the forward's per-pixel counts)")
    env_data = None if env is None else env.detach().contiguous()
    params = A.Params(levels, alpha, znear, background, flags & ~A.ADOP_FLAG_GRAD_ASSIGN, gamma, env_data)
    # Frames and workspace depend on the image sizes, not on the pose: they
    # are allocated first, while the GPU may still run the previous step;
    # reading a CUDA tangent below waits for it.
    dev = xyz.device
    frames = [A.Frame.alloc(c, feat.shape[1], levels, out_dtype, keep_state, dev,
                            xyz.shape[0] if keep_state else None) for c in cameras]
    sizing = A.Points(xyz.detach().contiguous(), feat.detach().contiguous(), None, radius, beta)
    ws = A.alloc_workspace(sizing, cameras, params, crf_luts, dev)
    cams = _effective_cameras(cameras, xi, intrinsics)
    outs = _Rasterize.apply(xyz, feat, xi, intrinsics, env, cams, params, out_dtype, keep_state, crf_luts,
                            (radius, beta), (frames, ws))
    return [list(outs[k * levels:(k + 1) * levels]) for k in range(len(cameras))]
