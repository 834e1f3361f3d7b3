"""Thin ctypes binding of ``include/adop.h``: the same entry points, with
torch CUDA tensors in place of raw device pointers.  Argument marshalling
only -- every step of the rasterizer runs in the CUDA library, and nothing
here falls back to another implementation: if ``libadop.so`` is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass, field

import numpy as np

from . import _build

ADOP_MAX_LEVELS = 8
ADOP_MAX_CAMERAS = 64
ADOP_FLAG_NORMAL_CULL = 1 << 0
ADOP_FLAG_GRAD_ALL_PROJECTED = 1 << 1
ADOP_FLAG_EPILOGUE = 1 << 2
ADOP_FLAG_GRAD_ASSIGN = 1 << 3
ADOP_FLAG_DISCARD = 1 << 4
ADOP_FLAG_LEAKY_CRF = 1 << 5
ADOP_FLAG_LOG_DESCRIPTORS = 1 << 6
ADOP_F32, ADOP_BF16, ADOP_F16 = 0, 1, 2

STATUS = {0: "ADOP_OK", 1: "ADOP_ERR_INVALID_ARG", 2: "ADOP_ERR_UNSUPPORTED", 3: "ADOP_ERR_OUT_OF_MEMORY",
          4: "ADOP_ERR_CUDA", 5: "ADOP_ERR_TIMEOUT", 6: "ADOP_ERR_BUSY", 7: "ADOP_ERR_CANCELLED"}


class AdopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class adop_intrinsics(ct.Structure):
    _fields_ = [("w", ct.c_int32), ("h", ct.c_int32)] + [
        (k, ct.c_float) for k in ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")] + [("model", ct.c_int32)]


class adop_pose(ct.Structure):
    _fields_ = [("R", ct.c_float * 9), ("t", ct.c_float * 3)]


class adop_photometric(ct.Structure):
    _fields_ = [("ev", ct.c_float), ("wb", ct.c_float * 3), ("vig_c", ct.c_float * 2), ("vig_a", ct.c_float * 3),
                ("crf_lut", ct.c_void_p), ("crf_n", ct.c_int32), ("enabled", ct.c_int32)]


class adop_camera(ct.Structure):
    _fields_ = [("K", adop_intrinsics), ("T", adop_pose), ("ph", adop_photometric)]


class adop_points(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("c", ct.c_int32), ("feat_dtype", ct.c_int32), ("xyz", ct.c_void_p),
                ("feat", ct.c_void_p), ("normals", ct.c_void_p), ("radius", ct.c_void_p), ("beta", ct.c_void_p)]


class adop_params(ct.Structure):
    _fields_ = [("levels", ct.c_int32), ("alpha", ct.c_float), ("znear", ct.c_float), ("background", ct.c_void_p),
                ("flags", ct.c_uint32), ("gamma", ct.c_float), ("env", ct.c_void_p), ("env_w", ct.c_int32),
                ("env_h", ct.c_int32), ("grad_dtype", ct.c_int32), ("grad_feat_dtype", ct.c_int32)]


class adop_frame(ct.Structure):
    _fields_ = [("image", ct.c_void_p * ADOP_MAX_LEVELS), ("key", ct.c_void_p * ADOP_MAX_LEVELS),
                ("count", ct.c_void_p * ADOP_MAX_LEVELS), ("acc", ct.c_void_p), ("vis", ct.c_void_p),
                ("out_dtype", ct.c_int32)]


class adop_kernel_stat(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int64), ("total_ms", ct.c_double)]


_P = ct.c_void_p
_lib = None

# (name, restype, argtypes) of every exported symbol of include/adop.h
SIGNATURES = {
    "adop_workspace_bytes": (ct.c_size_t, [_P, _P, ct.c_int32, _P]),
    "adop_render_forward": (ct.c_int, [_P, _P, ct.c_int32, _P, _P, _P, ct.c_size_t, _P]),
    "adop_render_backward": (ct.c_int, [_P, _P, ct.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, ct.c_size_t, _P]),
    "adop_last_error": (ct.c_char_p, []),
    "adop_abi_version": (ct.c_int32, []),
    "adop_render_backward_noalloc": (ct.c_int, [_P, _P, ct.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "adop_point_radius_workspace_bytes": (ct.c_size_t, [ct.c_int64]),
    "adop_point_radius": (ct.c_int, [_P, ct.c_int64, ct.c_int32, _P, _P, ct.c_size_t, _P]),
    "adop_env_backward": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32, _P, _P, _P, _P]),
    "adop_photometric_workspace_bytes": (ct.c_size_t, [ct.c_int32]),
    "adop_photometric_backward": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32, _P, _P, _P, _P, _P, ct.c_size_t, _P]),
    "adop_atomic_probe": (ct.c_int, [ct.c_int32, _P, ct.c_int64, ct.c_int64, ct.c_uint64, _P]),
    "adop_profile_enable": (ct.c_int, [ct.c_int32]),
    "adop_profile_collect": (ct.c_int32, [_P, ct.c_int32]),
    "adop_pose_apply_tangent": (ct.c_int, [_P, _P, ct.c_int32]),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load ``libadop.so`` (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run build())")
        lib = ct.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int):
    if st != 0:
        raise AdopError(st, load().adop_last_error().decode())


def _dev_ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _torch():
    import torch
    return torch


def dtype_code(dt) -> int:
    torch = _torch()
    if dt == torch.float32:
        return ADOP_F32
    if dt == torch.bfloat16:
        return ADOP_BF16
    if dt == torch.float16:
        return ADOP_F16
    raise ValueError(f"unsupported dtype {dt}")


@dataclass
class Points:
    """The point cloud: xyz (n x 3 float32), feat (n x c float32/bfloat16/float16),
    optional normals, and for stochastic discarding a world radius and a
    uniform draw per point (float32, n each)."""
    xyz: object
    feat: object
    normals: object = None
    radius: object = None
    beta: object = None

    def struct(self) -> adop_points:
        n, c = self.feat.shape
        assert tuple(self.xyz.shape) == (n, 3)
        return adop_points(n, c, dtype_code(self.feat.dtype), _dev_ptr(self.xyz), _dev_ptr(self.feat),
                           _dev_ptr(self.normals), _dev_ptr(self.radius), _dev_ptr(self.beta))


@dataclass
class Params:
    levels: int = 4
    alpha: float = 0.01
    znear: float = 1e-3
    background: object = None  # c float32 CUDA tensor or None
    flags: int = 0
    gamma: float = 1.5         # stochastic discarding (with ADOP_FLAG_DISCARD)
    env: object = None         # env_h x env_w x c float32 CUDA tensor (environment map) or None

    def struct(self) -> adop_params:
        eh, ew = (0, 0) if self.env is None else (int(self.env.shape[0]), int(self.env.shape[1]))
        return adop_params(self.levels, self.alpha, self.znear, _dev_ptr(self.background), self.flags, self.gamma,
                           _dev_ptr(self.env), ew, eh)


def camera_struct(cam, crf_lut=None) -> adop_camera:
    """Marshal a camera (attributes w, h, fx, fy, cx, cy, k1, k2, k3, p1, p2, R,
    t; optionally ev, wb, vig_c, vig_a and epilogue) into adop_camera.
    crf_lut: 3 x n float32 CUDA tensor of the response curve, or None."""
    K = adop_intrinsics(int(cam.w), int(cam.h), *[float(getattr(cam, k, 0.0)) for k in
                                                  ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")],
                        int(getattr(cam, "model", 0)))
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    T = adop_pose((ct.c_float * 9)(*R.tolist()), (ct.c_float * 3)(*t.tolist()))
    ph = adop_photometric(
        float(getattr(cam, "ev", 0.0)), (ct.c_float * 3)(*[float(v) for v in getattr(cam, "wb", (1, 1, 1))]),
        (ct.c_float * 2)(*[float(v) for v in getattr(cam, "vig_c", (0.5, 0.5))]),
        (ct.c_float * 3)(*[float(v) for v in getattr(cam, "vig_a", (0, 0, 0))]),
        _dev_ptr(crf_lut), 0 if crf_lut is None else int(crf_lut.shape[-1]),
        1 if getattr(cam, "epilogue", False) else 0)
    return adop_camera(K, T, ph)


def pyramid_offsets(w: int, h: int, levels: int):
    off = [0]
    for l in range(levels):
        off.append(off[-1] + (w >> l) * (h >> l))
    return off


@dataclass
class Frame:
    """One camera's outputs and per-pixel state (torch tensors)."""
    images: list
    key: object = None     # int64 (bit pattern of uint64), all layers concatenated
    count: object = None   # int32 (bit pattern of uint32)
    acc: object = None     # float32, pixel-major sums
    vis: object = None     # int32 per point: layer mask (bits 0-7) | screen tile << 8
    w: int = 0
    h: int = 0
    levels: int = 0
    keep: list = field(default_factory=list)

    @staticmethod
    def alloc(cam, c: int, levels: int, out_dtype=None, keep_state: bool = True, device="cuda",
              n_points: int | None = None):
        """Images of every layer; with keep_state also key/count/acc, and the
        per-point layer mask if n_points is given."""
        torch = _torch()
        out_dtype = out_dtype or torch.float32
        w, h = int(cam.w), int(cam.h)
        images = [torch.empty((c, h >> l, w >> l), dtype=out_dtype, device=device) for l in range(levels)]
        f = Frame(images, w=w, h=h, levels=levels)
        if keep_state:
            px = pyramid_offsets(w, h, levels)[-1]
            f.key = torch.empty(px, dtype=torch.int64, device=device)
            f.count = torch.empty(px, dtype=torch.int32, device=device)
            f.acc = torch.empty(px * c, dtype=torch.float32, device=device)
            if n_points is not None:
                f.vis = torch.empty(max(1, n_points), dtype=torch.int32, device=device)
        return f

    def layer(self, buf, l):
        off = pyramid_offsets(self.w, self.h, self.levels)
        return buf[off[l]:off[l + 1]].view(self.h >> l, self.w >> l)

    def struct(self) -> adop_frame:
        fr = adop_frame()
        off = pyramid_offsets(self.w, self.h, self.levels)
        for l, im in enumerate(self.images):
            fr.image[l] = _dev_ptr(im)
        if self.key is not None:
            for l in range(self.levels):
                fr.key[l] = self.key.data_ptr() + 8 * off[l]
                fr.count[l] = self.count.data_ptr() + 4 * off[l]
            fr.acc = self.acc.data_ptr()
            fr.vis = None if self.vis is None else self.vis.data_ptr()
        fr.out_dtype = dtype_code(self.images[0].dtype) if self.images else ADOP_F32
        return fr


def _cams_array(cams, crf_luts=None):
    arr = (adop_camera * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = camera_struct(cam, None if crf_luts is None else crf_luts[k])
    return arr


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def adop_pose_apply_tangent(xi, R, t):
    """exp(xi) (R, t) for one pose (Eq. tangent), computed by the library:
    xi = (nu, omega) (6 numbers), R (3 x 3) and t (3) -> (R', t') as float32
    numpy arrays."""
    x = np.ascontiguousarray(np.asarray(xi, np.float64).reshape(6))
    pose = adop_pose((ct.c_float * 9)(*np.asarray(R, np.float32).reshape(9).tolist()),
                     (ct.c_float * 3)(*np.asarray(t, np.float32).reshape(3).tolist()))
    _check(load().adop_pose_apply_tangent(x.ctypes.data_as(ct.c_void_p), ct.byref(pose), 1))
    return (np.array(pose.R[:], np.float32).reshape(3, 3), np.array(pose.t[:], np.float32))


def adop_abi_version() -> int:
    return int(load().adop_abi_version())


def adop_profile_enable(on: bool = True) -> None:
    _check(load().adop_profile_enable(1 if on else 0))


def adop_profile_collect() -> dict:
    """{kernel name: (launches, total device ms)} since the last collect."""
    lib = load()
    buf = (adop_kernel_stat * 64)()
    m = lib.adop_profile_collect(buf, 64)
    if m < 0:
        raise AdopError(4, lib.adop_last_error().decode())
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(m)}


def adop_last_error() -> str:
    return load().adop_last_error().decode()


def adop_workspace_bytes(points: Points, cams, params: Params, crf_luts=None) -> int:
    lib = load()
    ps, pr = points.struct(), params.struct()
    arr = _cams_array(cams, crf_luts)
    n = lib.adop_workspace_bytes(ct.byref(ps), arr, len(cams), ct.byref(pr))
    if n == 0:
        raise AdopError(1, lib.adop_last_error().decode())
    return int(n)


def alloc_workspace(points: Points, cams, params: Params, crf_luts=None, device="cuda"):
    torch = _torch()
    nbytes = adop_workspace_bytes(points, cams, params, crf_luts)
    return torch.empty(nbytes + 256, dtype=torch.uint8, device=device)


def _ws_ptr(ws):
    """256-byte aligned pointer and usable size of a workspace tensor."""
    p = ws.data_ptr()
    a = (p + 255) // 256 * 256
    return ct.c_void_p(a), ws.numel() - (a - p)


def adop_point_radius(xyz, k: int = 4, stream=None):
    """Distance of every point to its k-th nearest other point (float32 CUDA
    tensor), the world radius of stochastic point discarding (Sec. 3.1)."""
    torch = _torch()
    lib = load()
    n = xyz.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=xyz.device)
    nb = int(lib.adop_point_radius_workspace_bytes(n))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=xyz.device)
    wp, wn = _ws_ptr(ws)
    _check(lib.adop_point_radius(_dev_ptr(xyz.contiguous()), n, int(k), _dev_ptr(out), wp, wn, _stream_ptr(stream)))
    return out


def adop_photometric_backward(cams, params: Params, c: int, frames, grad_image0, grad_photo, grad_crf=None,
                              stream=None, crf_luts=None):
    """Gradients of the photometric parameters (Sec. 3.3), accumulated into
    grad_photo (n_cam x 9: ev, wb[3], vig_c[2], vig_a[3]) and grad_crf (the
    LUTs' gradients, camera after camera) from dL/d(layer-0 image)."""
    torch = _torch()
    g1, _ = _grad_image_ptrs([[g] for g in grad_image0], cams, 1, c, fp32_only=True)
    g0 = (ct.c_void_p * len(cams))(*[g1[k] for k in range(len(cams))])
    lib = load()
    pr = params.struct()
    arr = _cams_array(cams, crf_luts)
    fr = (adop_frame * len(frames))(*[f.struct() for f in frames])
    nb = int(lib.adop_photometric_workspace_bytes(len(cams)))
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=grad_photo.device)
    wp, wn = _ws_ptr(ws)
    _check(lib.adop_photometric_backward(arr, len(cams), ct.byref(pr), int(c), fr, g0, _dev_ptr(grad_photo),
                                         _dev_ptr(grad_crf), wp, wn, _stream_ptr(stream)))


def adop_atomic_probe(kind: int, buf, elems: int, ops: int, seed: int = 0, stream=None):
    """Launch `ops` random atomics of one kind into buf (measurement aid, see include/adop.h)."""
    _check(load().adop_atomic_probe(int(kind), _dev_ptr(buf), int(elems), int(ops), int(seed), _stream_ptr(stream)))


def adop_env_backward(cams, params: Params, c: int, frames, grad_images, grad_env, stream=None, crf_luts=None):
    """Gradient of the environment map params.env (Sec. 3.1), accumulated into
    grad_env (same shape) from grad_images[k][l] (dL/dI of camera k, layer l)
    at the pixels where no point landed."""
    gi, _ = _grad_image_ptrs(grad_images, cams, params.levels, c, fp32_only=True)
    lib = load()
    pr = params.struct()
    arr = _cams_array(cams, crf_luts)
    fr = (adop_frame * len(frames))(*[f.struct() for f in frames])
    _check(lib.adop_env_backward(arr, len(cams), ct.byref(pr), int(c), fr, gi, _dev_ptr(grad_env),
                                 _stream_ptr(stream)))


def _grad_image_ptrs(grad_images, cams, levels: int, c: int, fp32_only: bool = False):
    """Pointer array grad_image[k * levels + l] of the backward entry points
    and the gradients' storage type (the adop_dtype code; FP32 if none is
    given).  The kernels read each given gradient as c x h_l x w_l values of
    one type -- float32, or bfloat16 / float16 where the call takes them -- so
    anything else (another dtype, mixed dtypes, another size) is refused
    here, before any launch."""
    torch = _torch()
    gptr = (ct.c_void_p * (len(cams) * levels))()
    dt = None
    allowed = (torch.float32,) if fp32_only else (torch.float32, torch.bfloat16, torch.float16)
    given = []
    for k, cam in enumerate(cams):
        row = grad_images[k] if grad_images is not None else None
        for l in range(levels):
            g = row[l] if row is not None else None
            if g is None:
                continue
            if g.dtype not in allowed:
                raise ValueError(f"grad_images[{k}][{l}] must be {' or '.join(str(a) for a in allowed)}, got {g.dtype}")
            if dt is not None and g.dtype != dt:
                raise ValueError(f"grad_images mix {dt} and {g.dtype}: one storage type per call")
            dt = g.dtype
            want = c * (int(cam.h) >> l) * (int(cam.w) >> l)
            if g.numel() != want:
                raise ValueError(f"grad_images[{k}][{l}] has {g.numel()} elements, c x h_l x w_l = {want} expected")
            given.append((k * levels + l, g))
    for j, g in given:  # every check passed: marshal
        gptr[j] = _dev_ptr(g)
    return gptr, (ADOP_F32 if dt is None else dtype_code(dt))


def adop_render_forward(points: Points, cams, params: Params, frames, workspace, stream=None, crf_luts=None):
    """Forward pass (Sec. 3.1) of every camera; fills each frame's images and state."""
    lib = load()
    ps, pr = points.struct(), params.struct()
    arr = _cams_array(cams, crf_luts)
    fr = (adop_frame * len(frames))(*[f.struct() for f in frames])
    wp, wn = _ws_ptr(workspace)
    _check(lib.adop_render_forward(ct.byref(ps), arr, len(cams), ct.byref(pr), fr, wp, wn, _stream_ptr(stream)))


def adop_render_backward(points: Points, cams, params: Params, frames, grad_images, grad_feat=None,
                         grad_xyz=None, grad_pose=None, grad_intr=None, workspace=None, stream=None,
                         crf_luts=None):
    """Backward pass (Sec. 3.1).  grad_images[k][l]: dL/dI of camera k, layer l
    (CUDA tensor c x h_l x w_l or None; float32, bfloat16 or float16, one type
    per call).  grad_feat: float32, or bfloat16 / float16 with
    ADOP_FLAG_GRAD_ASSIGN and one camera (summed in FP32, rounded once)."""
    gptr, gdt = _grad_image_ptrs(grad_images, cams, params.levels, points.feat.shape[1])
    lib = load()
    ps, pr = points.struct(), params.struct()
    pr.grad_dtype = gdt
    pr.grad_feat_dtype = ADOP_F32 if grad_feat is None else dtype_code(grad_feat.dtype)
    arr = _cams_array(cams, crf_luts)
    fr = (adop_frame * len(frames))(*[f.struct() for f in frames])
    wp, wn = _ws_ptr(workspace)
    _check(lib.adop_render_backward(ct.byref(ps), arr, len(cams), ct.byref(pr), fr, gptr, _dev_ptr(grad_feat),
                                    _dev_ptr(grad_xyz), _dev_ptr(grad_pose), _dev_ptr(grad_intr), wp, wn,
                                    _stream_ptr(stream)))


def adop_render_backward_noalloc(points: Points, cams, params: Params, frames, grad_images, grad_feat=None,
                                 grad_xyz=None, grad_pose=None, grad_intr=None, stream=None, crf_luts=None):
    """adop_render_backward without a workspace: the library's static scratch
    array is used instead (for callers that may not allocate device memory).
    Frames must carry the forward's kept state."""
    gptr, gdt = _grad_image_ptrs(grad_images, cams, params.levels, points.feat.shape[1])
    lib = load()
    ps, pr = points.struct(), params.struct()
    pr.grad_dtype = gdt
    pr.grad_feat_dtype = ADOP_F32 if grad_feat is None else dtype_code(grad_feat.dtype)
    arr = _cams_array(cams, crf_luts)
    fr = (adop_frame * len(frames))(*[f.struct() for f in frames])
    _check(lib.adop_render_backward_noalloc(ct.byref(ps), arr, len(cams), ct.byref(pr), fr, gptr,
                                            _dev_ptr(grad_feat), _dev_ptr(grad_xyz), _dev_ptr(grad_pose),
                                            _dev_ptr(grad_intr), _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# render server (adop_serve_*)
# ---------------------------------------------------------------------------

class adop_serve_config(ct.Structure):
    _fields_ = [("mem_budget_bytes", ct.c_size_t), ("max_slots", ct.c_int32), ("streams", ct.c_int32),
                ("max_batch", ct.c_int32), ("levels", ct.c_int32), ("alpha", ct.c_float), ("znear", ct.c_float),
                ("flags", ct.c_uint32), ("out_dtype", ct.c_int32), ("background", ct.c_void_p),
                ("env", ct.c_void_p), ("env_w", ct.c_int32), ("env_h", ct.c_int32),
                ("batch_window_us", ct.c_int32)]


class adop_serve_stats(ct.Structure):
    _fields_ = [(k, ct.c_int64) for k in ("submitted", "completed", "cancelled", "failed", "queued", "active",
                                          "batches")] + \
               [(k, ct.c_double) for k in ("mean_batch", "p50_ms", "p99_ms", "mean_ms", "max_ms", "req_per_s",
                                           "points_per_s")] + \
               [("mem_in_use", ct.c_size_t), ("mem_peak", ct.c_size_t), ("mixed_batches", ct.c_int64)]


SIGNATURES.update({
    "adop_serve_create": (ct.c_int, [_P, _P]),
    "adop_serve_load_cloud": (ct.c_int, [_P, _P, _P]),
    "adop_serve_submit": (ct.c_int, [_P, ct.c_int32, _P, _P, _P]),
    "adop_serve_poll": (ct.c_int, [_P, ct.c_uint64]),
    "adop_serve_wait": (ct.c_int, [_P, ct.c_uint64, ct.c_int32]),
    "adop_serve_cancel": (ct.c_int, [_P, ct.c_uint64]),
    "adop_serve_latency": (ct.c_int, [_P, ct.c_uint64, _P]),
    "adop_serve_get_stats": (ct.c_int, [_P, _P]),
    "adop_serve_reset_stats": (ct.c_int, [_P]),
    "adop_serve_destroy": (ct.c_int, [_P]),
})


def output_numel(cam, c: int, levels: int) -> int:
    """Elements of a server output buffer: all layers, c x h_l x w_l each."""
    return c * pyramid_offsets(int(cam.w), int(cam.h), levels)[-1]


def split_output(buf, cam, c: int, levels: int):
    """Views of a server output buffer per layer (c x h_l x w_l)."""
    off = pyramid_offsets(int(cam.w), int(cam.h), levels)
    return [buf[c * off[l]:c * off[l + 1]].view(c, int(cam.h) >> l, int(cam.w) >> l) for l in range(levels)]


class Server:
    """Continuous-batching render server over adop_serve_* (see include/adop.h)."""

    def __init__(self, mem_budget_bytes: int, max_slots: int = 64, streams: int = 4, max_batch: int = 8,
                 levels: int = 4, alpha: float = 0.01, znear: float = 1e-3, flags: int = 0, out_dtype=None,
                 background=None, env=None, batch_window_us: int = 0):
        torch = _torch()
        self.lib = load()
        self.levels = levels
        self.out_dtype = out_dtype or torch.float32
        self._keep = {}
        self._clouds = []
        self._bg = background
        self._env = env
        eh, ew = (0, 0) if env is None else (int(env.shape[0]), int(env.shape[1]))
        cfg = adop_serve_config(mem_budget_bytes, max_slots, streams, max_batch, levels, alpha, znear, flags,
                                dtype_code(self.out_dtype), _dev_ptr(background), _dev_ptr(env), ew, eh,
                                int(batch_window_us))
        h = ct.c_void_p()
        _check(self.lib.adop_serve_create(ct.byref(cfg), ct.byref(h)))
        self.h = h

    def load_cloud(self, points: Points) -> int:
        ps = points.struct()
        cid = ct.c_int32()
        _check(self.lib.adop_serve_load_cloud(self.h, ct.byref(ps), ct.byref(cid)))
        self._clouds.append(points)
        return cid.value

    def submit(self, cloud_id: int, cam, out, crf_lut=None) -> int:
        cs = camera_struct(cam, crf_lut)
        t = ct.c_uint64()
        _check(self.lib.adop_serve_submit(self.h, cloud_id, ct.byref(cs), _dev_ptr(out), ct.byref(t)))
        self._keep[t.value] = (out, crf_lut)
        return t.value

    def poll(self, ticket: int) -> int:
        return int(self.lib.adop_serve_poll(self.h, ticket))

    def wait(self, ticket: int, timeout_ms: int = 60_000) -> int:
        st = int(self.lib.adop_serve_wait(self.h, ticket, timeout_ms))
        if st != 6 and st != 5:
            self._keep.pop(ticket, None)
        return st

    def cancel(self, ticket: int) -> int:
        return int(self.lib.adop_serve_cancel(self.h, ticket))

    def latency_ms(self, ticket: int) -> float:
        v = ct.c_double()
        _check(self.lib.adop_serve_latency(self.h, ticket, ct.byref(v)))
        return v.value

    def stats(self) -> dict:
        s = adop_serve_stats()
        _check(self.lib.adop_serve_get_stats(self.h, ct.byref(s)))
        return {k: getattr(s, k) for k, _ in adop_serve_stats._fields_}

    def reset_stats(self):
        _check(self.lib.adop_serve_reset_stats(self.h))

    def close(self):
        if self.h:
            _check(self.lib.adop_serve_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
