"""Plain FP64 CPU oracle of ADOP's one-pixel point rasterizer (Sec. 3.1, 3.3).

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import it.  It shares no code with
``paper_2110_06635_gb300`` and imports nothing from it; cameras and scenes are
read by duck typing (attributes ``w, h, fx, fy, cx, cy, k1, k2, k3, p1, p2, R,
t``), so the seeded generators in ``scenes`` can feed both sides.

The arithmetic lives in ``adop_oracle.c`` (compiled with ``-ffp-contract=off``
so that the FP32 projection contract is evaluated one IEEE operation at a
time).  This module only marshals numpy arrays.  A pure-Python list-based
brute-force renderer (``bruteforce``) restates Eq. blend and Eq. spatialderiv
with explicit per-pixel point lists, for tiny scenes.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adop_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fno-math-errno",
             "-Wall"]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, no FMA
    contraction), with OpenMP where the compiler has it (threads are a timing
    aid only: the results do not depend on them), else without."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", *GCC_FLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Intr(ct.Structure):
    _fields_ = [("w", ct.c_int32), ("h", ct.c_int32)] + [
        (k, ct.c_float) for k in ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")] + [("model", ct.c_int32)]


class _Pose(ct.Structure):
    _fields_ = [("R", ct.c_float * 9), ("t", ct.c_float * 3)]


_P = ct.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ct.CDLL(build())
        lib.orc_project_f32.argtypes = [_P, _P, _P, _P, _P, _P]
        lib.orc_project_f32.restype = ct.c_int
        lib.orc_camera_fisheye_f64.argtypes = [_P, _P, _P]
        lib.orc_pixel.argtypes = [ct.c_float, ct.c_float, ct.c_int, ct.c_int32, ct.c_int32, _P, _P]
        lib.orc_pixel.restype = ct.c_int
        lib.orc_pyramid_pixels.argtypes = [ct.c_int32, ct.c_int32, ct.c_int]
        lib.orc_pyramid_pixels.restype = ct.c_int64
        lib.orc_forward.argtypes = [ct.c_int64, _P, ct.c_int32, _P, _P, _P, _P, ct.c_int32, ct.c_float,
                                    ct.c_float, _P, _P, _P, ct.c_float, ct.c_int32, _P, ct.c_int32, ct.c_int32,
                                    _P, _P, _P, _P, _P, ct.c_int32]
        lib.orc_threads.argtypes = [ct.c_int32]
        lib.orc_threads.restype = ct.c_int32
        lib.orc_camera_inverse_f64.argtypes = [_P, ct.c_double, ct.c_double, _P]
        lib.orc_env_sample.argtypes = [_P, ct.c_int32, ct.c_int32, ct.c_int32, _P, _P, _P, _P]
        lib.orc_env_grad.argtypes = [_P, _P, ct.c_int32, ct.c_int32, _P, _P, ct.c_int32, ct.c_int32, _P]
        lib.orc_knn_radius.argtypes = [ct.c_int64, _P, ct.c_int32, _P]
        lib.orc_forward.restype = ct.c_int
        lib.orc_project_jac_f64.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        lib.orc_camera_f64.argtypes = [_P, _P, _P]
        lib.orc_camera_f64_many.argtypes = [ct.c_int64, _P, _P, _P, ct.c_int32]
        lib.orc_backward.argtypes = [ct.c_int64, _P, ct.c_int32, _P, _P, _P, ct.c_int32, ct.c_float,
                                     _P, ct.c_int32, ct.c_int32, _P, _P, _P, _P, _P, _P,
                                     _P, _P, _P, _P, _P, _P, _P, _P, _P, ct.c_int64, ct.c_int32]
        lib.orc_backward.restype = ct.c_int
        lib.orc_epilogue.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, _P, ct.c_double, _P, _P, _P,
                                     _P, ct.c_int32, ct.c_int32, _P]
        lib.orc_photometric_grad.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, _P, _P, ct.c_double, _P, _P, _P,
                                             _P, ct.c_int32, ct.c_int32, _P, _P, _P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _intr(cam) -> _Intr:
    return _Intr(int(cam.w), int(cam.h), *[float(getattr(cam, k)) for k in
                                           ("fx", "fy", "cx", "cy", "k1", "k2", "k3", "p1", "p2")],
                 int(getattr(cam, "model", 0)))


def _pose(cam) -> _Pose:
    R = np.ascontiguousarray(np.asarray(cam.R, dtype=np.float32).reshape(9))
    t = np.ascontiguousarray(np.asarray(cam.t, dtype=np.float32).reshape(3))
    return _Pose((ct.c_float * 9)(*R.tolist()), (ct.c_float * 3)(*t.tolist()))


def layer_shapes(w: int, h: int, levels: int):
    """(h_l, w_l) of each pyramid layer: w_l = w >> l, h_l = h >> l."""
    return [(h >> l, w >> l) for l in range(levels)]


def split_layers(flat: np.ndarray, w: int, h: int, levels: int, c: int | None = None):
    """Split a concatenated per-layer array into a list (planar c x h_l x w_l if c)."""
    out, off = [], 0
    for hl, wl in layer_shapes(w, h, levels):
        n = hl * wl * (c or 1)
        blk = flat[off:off + n]
        out.append(blk.reshape((c, hl, wl) if c else (hl, wl)))
        off += n
    return out


def project_f32(cam, x):
    """FP32 projection contract for one point -> (u0, v0, z) as numpy float32."""
    lib = _load()
    xv = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(3))
    out = np.zeros(3, dtype=np.float32)
    K, T = _intr(cam), _pose(cam)
    lib.orc_project_f32(ct.byref(K), ct.byref(T), _ptr(xv), _ptr(out[0:]), _ptr(out[1:]), _ptr(out[2:]))
    return out[0], out[1], out[2]


def pixel(u0, v0, l, w, h):
    """Eq. round + Eq. boundscheck at layer l -> (pu, pv) or None."""
    lib = _load()
    pu, pv = ct.c_int32(), ct.c_int32()
    ok = lib.orc_pixel(ct.c_float(u0), ct.c_float(v0), int(l), int(w), int(h), ct.byref(pu), ct.byref(pv))
    return (pu.value, pv.value) if ok else None


def project_jac_f64(cam, x):
    """FP64 (u0, v0), X, d(u0,v0)/dX (2x3) and d(u0,v0)/d(fx,fy,cx,cy,k1,k2) (2x6)."""
    lib = _load()
    xv = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(3))
    uv, X = np.zeros(2), np.zeros(3)
    JX, JK = np.zeros(6), np.zeros(12)
    K, T = _intr(cam), _pose(cam)
    lib.orc_project_jac_f64(ct.byref(K), ct.byref(T), _ptr(xv), _ptr(uv), _ptr(X), _ptr(JX), _ptr(JK))
    return uv, X, JX.reshape(2, 3), JK.reshape(2, 6)


def camera_fisheye_f64(k9, X):
    """The fisheye model (stereographic + radial polynomial) in FP64."""
    lib = _load()
    k = np.ascontiguousarray(k9, dtype=np.float64).reshape(9)
    Xv = np.ascontiguousarray(X, dtype=np.float64).reshape(3)
    uv = np.zeros(2)
    lib.orc_camera_fisheye_f64(_ptr(k), _ptr(Xv), _ptr(uv))
    return uv


def camera_f64(k9, X):
    """The camera model in FP64: k9 = (fx, fy, cx, cy, k1, k2, k3, p1, p2),
    X camera-space point -> (u0, v0)."""
    lib = _load()
    k = np.ascontiguousarray(k9, dtype=np.float64).reshape(9)
    Xv = np.ascontiguousarray(X, dtype=np.float64).reshape(3)
    uv = np.zeros(2)
    lib.orc_camera_f64(_ptr(k), _ptr(Xv), _ptr(uv))
    return uv


def camera_f64_many(k9, X, model=0):
    """camera_f64 (or the fisheye model) over an n x 3 array of camera-space points -> n x 2."""
    lib = _load()
    k = np.ascontiguousarray(k9, dtype=np.float64).reshape(9)
    Xv = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    uv = np.zeros((Xv.shape[0], 2))
    lib.orc_camera_f64_many(Xv.shape[0], _ptr(k), _ptr(Xv), _ptr(uv), int(model))
    return uv


@dataclass
class Forward:
    keys: np.ndarray   # uint64, concatenated pyramid
    cnt: np.ndarray    # uint32
    img: np.ndarray    # float64, concatenated planar c x h_l x w_l
    pix: np.ndarray    # int32 n x levels (-1 = discarded)
    z: np.ndarray      # float32 n
    w: int
    h: int
    levels: int
    c: int

    def layer_keys(self):
        return split_layers(self.keys, self.w, self.h, self.levels)

    def layer_cnt(self):
        return split_layers(self.cnt, self.w, self.h, self.levels)

    def layer_img(self):
        return split_layers(self.img, self.w, self.h, self.levels, self.c)


def feat_to_f64(feat) -> np.ndarray:
    """Exact upcast of stored features to FP64.  BF16 arrives as uint16 bit
    patterns (the upper half of an IEEE binary32), FP16 as numpy float16."""
    f = np.asarray(feat)
    if f.dtype == np.uint16:
        return (f.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return f.astype(np.float64)


def knn_radius(xyz, k: int = 4) -> np.ndarray:
    """Distance to the k-th nearest other point (FP64, exhaustive; small clouds)."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    out = np.empty(xyz.shape[0])
    lib.orc_knn_radius(xyz.shape[0], _ptr(xyz), int(k), _ptr(out))
    return out


def threads(requested: int = 0) -> int:
    """Threads a request gets (0: every core; 1 without OpenMP)."""
    return int(_load().orc_threads(int(requested)))


def forward(xyz, feat, cam, levels=4, alpha=0.01, znear=1e-3, background=None, normals=None,
            radius=None, beta=None, gamma=1.5, log_desc=False, env=None, threads=1) -> Forward:
    """One camera through Sec. 3.1's forward pass (Eq. render ... Eq. blend);
    with radius/beta, stochastic point discarding (Eq. discard) at every layer.
    threads (0 = every core) changes the time, not the result."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    f64 = np.ascontiguousarray(feat_to_f64(feat))
    n, c = f64.shape
    assert xyz.shape == (n, 3)
    npx = int(lib.orc_pyramid_pixels(int(cam.w), int(cam.h), int(levels)))
    keys = np.empty(npx, dtype=np.uint64)
    cnt = np.empty(npx, dtype=np.uint32)
    img = np.empty(npx * c, dtype=np.float64)
    pix = np.empty((n, levels), dtype=np.int32)
    z = np.empty(n, dtype=np.float32)
    bg = None if background is None else np.ascontiguousarray(background, dtype=np.float64)
    nrm = None if normals is None else np.ascontiguousarray(normals, dtype=np.float32)
    rad = None if radius is None else np.ascontiguousarray(radius, dtype=np.float32)
    bet = None if radius is None else np.ascontiguousarray(beta, dtype=np.float32)
    K, T = _intr(cam), _pose(cam)
    E = None if env is None else np.ascontiguousarray(env, dtype=np.float64)
    eh, ew = (0, 0) if env is None else E.shape[1:]
    rc = lib.orc_forward(n, _ptr(xyz), c, _ptr(f64), _ptr(nrm), ct.byref(K), ct.byref(T), int(levels),
                         ct.c_float(alpha), ct.c_float(znear), _ptr(bg), _ptr(rad), _ptr(bet), ct.c_float(gamma),
                         int(bool(log_desc)), _ptr(E), ew, eh, _ptr(keys), _ptr(cnt), _ptr(img), _ptr(pix), _ptr(z),
                         int(threads))
    if rc != 0:
        raise MemoryError("oracle forward: allocation failed")
    return Forward(keys, cnt, img, pix, z, int(cam.w), int(cam.h), int(levels), c)


def keys_counts(xyz, cam, levels=4, alpha=0.01, znear=1e-3, threads=1) -> Forward:
    """Sec. 3.1's forward without descriptors: every point's pixel per layer
    and depth (Eq. render ... Eq. boundscheck), the nearest-depth keys and the
    fuzzy-test counts |Lambda| (Eq. depthtest) -- for clouds too large to
    blend in FP64 here.  ``img`` is empty."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    n = xyz.shape[0]
    npx = int(lib.orc_pyramid_pixels(int(cam.w), int(cam.h), int(levels)))
    keys = np.empty(npx, dtype=np.uint64)
    cnt = np.empty(npx, dtype=np.uint32)
    img = np.empty(1, dtype=np.float64)
    pix = np.empty((n, levels), dtype=np.int32)
    z = np.empty(n, dtype=np.float32)
    K, T = _intr(cam), _pose(cam)
    rc = lib.orc_forward(n, _ptr(xyz), 0, None, None, ct.byref(K), ct.byref(T), int(levels), ct.c_float(alpha),
                         ct.c_float(znear), None, None, None, ct.c_float(1.5), 0, None, 0, 0,
                         _ptr(keys), _ptr(cnt), _ptr(img), _ptr(pix), _ptr(z), int(threads))
    if rc != 0:
        raise MemoryError("oracle forward: allocation failed")
    return Forward(keys, cnt, img[:0], pix, z, int(cam.w), int(cam.h), int(levels), 0)


def camera_inverse(cam, u0, v0):
    """Unit camera-space direction of the ray through layer-0 coordinates (u0, v0)."""
    lib = _load()
    d = np.zeros(3)
    K = _intr(cam)
    lib.orc_camera_inverse_f64(ct.byref(K), float(u0), float(v0), _ptr(d))
    return d


def env_sample(env, direction):
    """Bilinear equirectangular lookup of a world direction in env (c x h x w)."""
    lib = _load()
    E = np.ascontiguousarray(env, dtype=np.float64)
    c, eh, ew = E.shape
    out = np.zeros(c)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    lib.orc_env_sample(_ptr(E), c, ew, eh, _ptr(d), _ptr(out), None, None)
    return out


def env_grad(fwd, cam, G, env_shape):
    """dL/dE of the environment map (c x h x w) from the forward's empty pixels."""
    lib = _load()
    c, eh, ew = env_shape
    dE = np.zeros((c, eh, ew))
    K, T = _intr(cam), _pose(cam)
    Gv = np.ascontiguousarray(G, dtype=np.float64)
    lib.orc_env_grad(ct.byref(K), ct.byref(T), fwd.levels, c, _ptr(fwd.cnt), _ptr(Gv), ew, eh, _ptr(dE))
    return dE


@dataclass
class Backward:
    dfeat: np.ndarray
    dxyz: np.ndarray
    dpose: np.ndarray
    dintr: np.ndarray
    dpose_abs: np.ndarray
    dintr_abs: np.ndarray
    gu: np.ndarray
    gv: np.ndarray


def backward(fwd: Forward, xyz, feat, cam, G, alpha=0.01, background=None, all_projected=False,
             log_desc=False, threads=1, sample=None, layer_grads=True) -> Backward:
    """Sec. 3.1's backward pass for one camera; G is dL/dI over the
    concatenated pyramid (same layout as ``fwd.img``).  sample: point indices
    to visit (None = all): only their rows are written and only their terms
    are summed into the pose and intrinsics gradients.  threads (0 = every
    core) changes the time; only the reduced sums' FP64 rounding may follow it."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    f64 = np.ascontiguousarray(feat_to_f64(feat))
    n, c = f64.shape
    G = np.ascontiguousarray(G, dtype=np.float64)
    assert G.shape == fwd.img.shape
    dfeat = np.empty((n, c))
    dxyz = np.empty((n, 3))
    dpose, dintr, dpa, dia = (np.empty(6) for _ in range(4))
    # the per-layer g_u, g_v (n x levels each) only when asked for: at 10^8 points they are GBs
    gu = np.empty((n, fwd.levels)) if layer_grads else None
    gv = np.empty((n, fwd.levels)) if layer_grads else None
    bg = None if background is None else np.ascontiguousarray(background, dtype=np.float64)
    smp = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    if smp is not None and smp.size and (smp.min() < 0 or smp.max() >= n):
        raise IndexError("sample index outside [0, n)")
    K, T = _intr(cam), _pose(cam)
    rc = lib.orc_backward(n, _ptr(xyz), c, _ptr(f64), ct.byref(K), ct.byref(T), fwd.levels,
                          ct.c_float(alpha), _ptr(bg), int(bool(all_projected)), int(bool(log_desc)), _ptr(fwd.keys),
                          _ptr(fwd.cnt), _ptr(fwd.img), _ptr(fwd.pix), _ptr(fwd.z), _ptr(G),
                          _ptr(dfeat), _ptr(dxyz), _ptr(dpose), _ptr(dintr), _ptr(dpa), _ptr(dia),
                          _ptr(gu), _ptr(gv), _ptr(smp), 0 if smp is None else smp.size, int(threads))
    if rc != 0:
        raise MemoryError("oracle backward: allocation failed")
    return Backward(dfeat, dxyz, dpose, dintr, dpa, dia, gu, gv)


def epilogue(img0, ev=0.0, wb=(1.0, 1.0, 1.0), vig_c=(0.5, 0.5), vig_a=(0.0, 0.0, 0.0), crf=None,
             want_grad=False, leaky=False):
    """Sec. 3.3 photometric model on a layer-0 image (c x h x w, FP64).
    Returns the new image (and d out / d in if want_grad).  leaky: the
    training response curve of Eq. resonseleak."""
    lib = _load()
    img = np.array(img0, dtype=np.float64, copy=True, order="C")
    c, h, w = img.shape
    grad = np.empty_like(img) if want_grad else None
    lut = None if crf is None else np.ascontiguousarray(crf, dtype=np.float64)
    crf_n = 0 if crf is None else lut.shape[-1]
    lib.orc_epilogue(w, h, c, _ptr(img), ct.c_double(ev), _ptr(np.asarray(wb, np.float64)),
                     _ptr(np.asarray(vig_c, np.float64)), _ptr(np.asarray(vig_a, np.float64)),
                     _ptr(lut), crf_n, int(bool(leaky)), _ptr(grad))
    return (img, grad) if want_grad else img


def photometric_grad(img0, G, ev=0.0, wb=(1.0, 1.0, 1.0), vig_c=(0.5, 0.5), vig_a=(0.0, 0.0, 0.0), crf=None,
                     leaky=False, with_abs=False):
    """dL/d(EV, wb[3], c_v[2], a2, a4, a6) and dL/dLUT (3 x n) of the photometric
    model (Sec. 3.3) on a layer-0 image before the epilogue, given dL/d(out)."""
    lib = _load()
    img = np.ascontiguousarray(img0, dtype=np.float64)
    Gv = np.ascontiguousarray(G, dtype=np.float64)
    c, h, w = img.shape
    lut = None if crf is None else np.ascontiguousarray(crf, dtype=np.float64)
    crf_n = 0 if crf is None else lut.shape[-1]
    gp, gabs = np.zeros(9), np.zeros(9)
    gcrf = np.zeros((3, max(crf_n, 1)))
    lib.orc_photometric_grad(w, h, c, _ptr(img), _ptr(Gv), ct.c_double(ev), _ptr(np.asarray(wb, np.float64)),
                             _ptr(np.asarray(vig_c, np.float64)), _ptr(np.asarray(vig_a, np.float64)), _ptr(lut),
                             crf_n, int(bool(leaky)), _ptr(gp), _ptr(gcrf) if crf_n else None, _ptr(gabs))
    out = (gp, (gcrf if crf_n else None))
    return out + (gabs,) if with_abs else out


from .bruteforce import bruteforce_render, bruteforce_spatial  # noqa: E402,F401
