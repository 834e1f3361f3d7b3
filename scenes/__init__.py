"""Seeded synthetic scenes and cameras for ADOP's rasterizer.

This module is the ONLY code that both the CUDA path's tests/benchmark and the
CPU oracle's tests consume.  It holds none of the rasterizer's arithmetic: no
projection, rounding, depth test, blending or gradient -- only geometry
sampling (points on planes and spheres), random features and upstream
gradients, camera placement (look-at poses, orbits) and storage conversions
(FP32 -> BF16 / FP16 bit patterns).

The paper's scenes (Table scenes: Tanks and Temples, Kemenate, Boat, Office;
9.7M-72.9M points, 1920x1080 to 5472x3648) are not available; these seeded
stand-ins reproduce their shape: millions to 100M+ surface points, depth
complexity of several surfaces per pixel, distorted pinhole cameras at 1080p
and 4K, 4 to 8 feature channels.  Points are written surface by surface, and
within a surface in blocked (tile-by-tile) order of a jittered grid, so that
neighbouring indices are neighbours in space, as in a scanned or MVS cloud
after the paper's locality-preserving shuffle.  ``shuffle=True`` permutes them.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

__all__ = ["Camera", "Scene", "look_at", "tiny_spheres", "surfaces_scene", "single_view_camera",
           "orbit_cameras", "upstream_grad", "to_bf16_bits", "bf16_bits_to_f32", "config"]


@dataclass
class Camera:
    """Distorted pinhole camera + world-to-camera pose (camera looks along +z,
    image y points down) + the per-image photometric parameters."""
    w: int
    h: int
    fx: float
    fy: float
    cx: float
    cy: float
    k1: float = 0.0
    k2: float = 0.0
    k3: float = 0.0
    p1: float = 0.0
    p2: float = 0.0
    R: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))
    ev: float = 0.0
    wb: tuple = (1.0, 1.0, 1.0)
    vig_c: tuple = (0.5, 0.5)
    vig_a: tuple = (0.0, 0.0, 0.0)
    crf: np.ndarray | None = None  # 3 x n LUT on [0,1] or None
    epilogue: bool = False         # apply the photometric model to this view
    model: int = 0                 # 0 pinhole + Brown-Conrady, 1 fisheye (stereographic)

    def with_pose(self, R, t) -> "Camera":
        return replace(self, R=np.asarray(R, np.float32), t=np.asarray(t, np.float32))


@dataclass
class Scene:
    xyz: np.ndarray          # n x 3 float32
    feat: np.ndarray         # n x c float32 (the draw; BF16/FP16 are derived from it)
    normals: np.ndarray | None = None
    surface_id: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def c(self) -> int:
        return int(self.feat.shape[1])

    def feat_as(self, dtype: str) -> np.ndarray:
        """Stored features: 'f32' float32, 'bf16' uint16 bit patterns, 'f16' float16."""
        if dtype == "f32":
            return self.feat
        if dtype == "bf16":
            return to_bf16_bits(self.feat)
        if dtype == "f16":
            return self.feat.astype(np.float16)
        raise ValueError(dtype)


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (nearest, ties to even) and return the uint16 bits."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(np.asarray(a, dtype=np.float32))
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    out = r.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


def look_at(eye, target, down=(0.0, 1.0, 0.0)):
    """World-to-camera (R, t) of a camera at `eye` looking at `target`; the
    image y axis points along `down` projected onto the image plane."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = -np.asarray(down, np.float64)
    x = np.cross(f, up)
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(f, np.array([1.0, 0.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    return R.astype(np.float32), t.astype(np.float32)


# ----------------------------------------------------------------------------
# point sampling
# ----------------------------------------------------------------------------

def _blocked_grid(gx: int, gy: int, block: int = 8):
    """Cell indices (ix, iy) of a gx x gy grid in tile-by-tile order."""
    iy, ix = np.meshgrid(np.arange(gy), np.arange(gx), indexing="ij")
    ix, iy = ix.ravel(), iy.ravel()
    key = (((iy // block) * ((gx + block - 1) // block) + ix // block) * block * block
           + (iy % block) * block + ix % block)
    order = np.argsort(key, kind="stable")
    return ix[order], iy[order]


def _jittered(rng, m: int, aspect: float):
    """m jittered samples in [0,1]^2 in blocked order (aspect = width/height)."""
    gx = max(1, int(np.ceil(np.sqrt(m * aspect))))
    gy = max(1, int(np.ceil(m / gx)))
    ix, iy = _blocked_grid(gx, gy)
    if ix.size > m:  # drop surplus cells uniformly, keep the order
        keep = np.sort(rng.choice(ix.size, size=m, replace=False))
        ix, iy = ix[keep], iy[keep]
    s = (ix + rng.random(m)) / gx
    t = (iy + rng.random(m)) / gy
    return s, t


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def _split_counts(n: int, weights) -> np.ndarray:
    w = np.asarray(weights, np.float64)
    raw = n * w / w.sum()
    cnt = np.floor(raw).astype(np.int64)
    rem = n - int(cnt.sum())
    cnt[np.argsort(-(raw - cnt), kind="stable")[:rem]] += 1
    return cnt


def _sphere_points(rng, m, center, radius):
    s, t = _jittered(rng, m, 2.0)          # (phi, z) cells of equal area
    phi = 2 * np.pi * s
    zc = 2 * t - 1
    rr = np.sqrt(np.maximum(0.0, 1 - zc * zc))
    nrm = np.stack([rr * np.cos(phi), rr * np.sin(phi), zc], axis=1)
    return center + radius * nrm, nrm


def _plane_points(rng, m, center, a, b, Rm):
    s, t = _jittered(rng, m, a / b)
    local = np.stack([(s - 0.5) * a, (t - 0.5) * b, np.zeros(m)], axis=1)
    nrm = np.broadcast_to(Rm[:, 2], (m, 3))
    return center + local @ Rm.T, np.array(nrm)


def _finish(rng, pts, nrm, sid, c, noise, shuffle, feat_rng):
    pts = pts + rng.normal(scale=noise, size=pts.shape) if noise > 0 else pts
    n = pts.shape[0]
    feat = feat_rng.standard_normal((n, c), dtype=np.float32)
    if shuffle:
        perm = rng.permutation(n)
        pts, nrm, sid, feat = pts[perm], nrm[perm], sid[perm], feat[perm]
    return Scene(np.ascontiguousarray(pts, np.float32), np.ascontiguousarray(feat, np.float32),
                 np.ascontiguousarray(nrm, np.float32), sid.astype(np.int32))


def tiny_spheres(n: int = 20000, c: int = 4, seed: int = 1001, shuffle: bool = False) -> Scene:
    """3 spheres, radius U(0.2, 0.5), centres U[0,1]^3, points uniform on the
    surfaces (split by area), N(0, 1e-3^2) noise, features N(0,1)."""
    rng = np.random.default_rng(seed)
    centers = rng.random((3, 3))
    radii = rng.uniform(0.2, 0.5, size=3)
    counts = _split_counts(n, radii ** 2)
    P, N, S = [], [], []
    for k in range(3):
        p, nn = _sphere_points(rng, int(counts[k]), centers[k], radii[k])
        P.append(p); N.append(nn); S.append(np.full(len(p), k))
    return _finish(rng, np.concatenate(P), np.concatenate(N), np.concatenate(S), c, 1e-3, shuffle,
                   np.random.default_rng(seed + 7919))


def surfaces_scene(n: int, c: int = 8, n_planes: int = 25, n_spheres: int = 25, box: float = 10.0,
                   seed: int = 1002, size_scale: float = 1.0, shuffle: bool = False,
                   noise: float = 1e-3) -> Scene:
    """Points on seeded planes (rectangles with sides U(1,6) m x size_scale,
    random orientation) and spheres (radius U(0.3, 2) m x size_scale) with
    centres uniform in a box of side `box` m centred at the origin; points
    split in proportion to area."""
    rng = np.random.default_rng(seed)
    half = box / 2
    shapes, areas = [], []
    for _ in range(n_planes):
        a, b = rng.uniform(1.0, 6.0, size=2) * size_scale * box / 10.0
        shapes.append(("plane", rng.uniform(-half, half, 3), a, b, _random_rotation(rng)))
        areas.append(a * b)
    for _ in range(n_spheres):
        r = rng.uniform(0.3, 2.0) * size_scale * box / 10.0
        shapes.append(("sphere", rng.uniform(-half, half, 3), r))
        areas.append(4 * np.pi * r * r)
    counts = _split_counts(n, areas)
    P = np.empty((n, 3)); N = np.empty((n, 3)); S = np.empty(n, np.int32)
    o = 0
    for k, shp in enumerate(shapes):
        m = int(counts[k])
        if m == 0:
            continue
        if shp[0] == "plane":
            p, nn = _plane_points(rng, m, shp[1], shp[2], shp[3], shp[4])
        else:
            p, nn = _sphere_points(rng, m, shp[1], shp[2])
        P[o:o + m] = p; N[o:o + m] = nn; S[o:o + m] = k
        o += m
    return _finish(rng, P, N, S, c, noise, shuffle, np.random.default_rng(seed + 7919))


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def crf_gamma_lut(n: int = 256, gamma: float = 0.45) -> np.ndarray:
    """The paper's initial response curve x^0.45 as a 3 x n LUT."""
    x = np.linspace(0.0, 1.0, n)
    return np.stack([x ** gamma] * 3).astype(np.float32)


def env_map(c: int, eh: int = 64, ew: int = 128, seed: int = 1006, noise: float = 0.05) -> np.ndarray:
    """A c x eh x ew FP32 equirectangular environment map: a few random
    low-frequency waves in longitude and colatitude (sky-like, smooth across
    the seam) plus a little per-texel noise, values around [0, 1]."""
    rng = np.random.default_rng(seed)
    phi = (np.arange(ew) + 0.5) / ew * 2 * np.pi - np.pi
    theta = (np.arange(eh) + 0.5) / eh * np.pi
    P, T = np.meshgrid(phi, theta)
    out = np.empty((c, eh, ew), np.float64)
    for ch in range(c):
        v = np.full_like(P, 0.5)
        for _ in range(4):
            a, b = rng.integers(1, 4), rng.integers(1, 4)
            v += rng.uniform(-0.15, 0.15) * np.cos(a * P + rng.uniform(0, 2 * np.pi)) * np.cos(b * T)
        out[ch] = v + noise * rng.standard_normal(P.shape)
    return out.astype(np.float32)


def tiny_camera() -> Camera:
    """256^2, fx = fy = 205, principal point at the centre, k1 = 0.01; at
    (0,0,-2) looking at the origin (R = I, t = (0,0,2))."""
    return Camera(256, 256, 205.0, 205.0, 128.0, 128.0, k1=0.01,
                  R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 2], np.float32))


def single_view_camera(w: int = 1920, h: int = 1080, seed: int = 1002, dist: float = 12.0,
                       f: float = 1500.0, k1: float = -0.05, k2: float = 0.01) -> Camera:
    """A camera `dist` m from the origin on a seeded direction, looking at it."""
    rng = np.random.default_rng(seed + 31)
    az = rng.uniform(0, 2 * np.pi)
    el = rng.uniform(-0.3, 0.3)
    eye = dist * np.array([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)])
    R, t = look_at(eye, np.zeros(3))
    return Camera(w, h, f, f, w / 2, h / 2, k1=k1, k2=k2, R=R, t=t)


def orbit_cameras(k: int = 16, seed: int = 1003, radius: float = 12.0,
                  resolutions=((960, 540), (1280, 720), (1600, 900), (1920, 1080)),
                  f_rel: float = 0.78, photometric: bool = True) -> list:
    """k cameras on a seeded circular orbit (radius jitter 5%, elevation
    jitter), each with its own resolution, EV ~ U(-1,1), white balance R,B ~
    U(0.8,1.2), vignette a = (-0.1, 0, 0) and the x^0.45 response curve."""
    rng = np.random.default_rng(seed)
    cams = []
    lut = crf_gamma_lut()
    for j in range(k):
        az = 2 * np.pi * j / k + rng.normal(scale=0.05)
        el = rng.uniform(-0.25, 0.25)
        rad = radius * (1 + rng.uniform(-0.05, 0.05))
        eye = rad * np.array([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)])
        R, t = look_at(eye, rng.normal(scale=0.3, size=3))
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        cam = Camera(w, h, f_rel * w, f_rel * w, w / 2, h / 2, k1=-0.05, k2=0.01, R=R, t=t)
        if photometric:
            cam.epilogue = True
            cam.ev = float(rng.uniform(-1, 1))
            cam.wb = (float(rng.uniform(0.8, 1.2)), 1.0, float(rng.uniform(0.8, 1.2)))
            cam.vig_a = (-0.1, 0.0, 0.0)
            cam.crf = lut
        cams.append(cam)
    return cams


def path_cameras(k: int, w: int, h: int, seed: int = 1004, radius: float = 60.0) -> list:
    """k cameras along a smooth seeded path around a large scene."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, size=3)
    cams = []
    for j in range(k):
        s = j / max(1, k)
        az = 2 * np.pi * 0.25 * s + ph[0]
        eye = np.array([radius * np.cos(az), 5 + 3 * np.sin(2 * np.pi * s + ph[1]), radius * np.sin(az)])
        tgt = np.array([5 * np.cos(2 * np.pi * s + ph[2]), 0.0, 5 * np.sin(2 * np.pi * s + ph[2])])
        R, t = look_at(eye, tgt)
        cams.append(Camera(w, h, 0.78 * w, 0.78 * w, w / 2, h / 2, k1=-0.05, k2=0.01, R=R, t=t))
    return cams


def upstream_grad(w: int, h: int, levels: int, c: int, seed: int) -> list:
    """N(0,1) dL/dI for each layer (c x h_l x w_l float32)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((c, h >> l, w >> l), dtype=np.float32) for l in range(levels)]


def config(k: int, n: int | None = None, shuffle: bool = False):
    """The standard workloads, by number:
      1  tiny: 20,000 points on 3 spheres, C = 4, one 256^2 camera
      2  single view: 5M points on 25 planes + 25 spheres in a 10 m box, C = 8,
         1920x1080 camera 12 m from the centre, fx = fy = 1500, k1 = -0.05, k2 = 0.01
      3  training step: 20M points, C = 8, 16 orbit cameras 960x540..1920x1080
      4  large scene: 120M points on 500 surfaces in a 100 m box, C = 4
    Returns (scene, cameras).  `n` overrides the point count (subsamples)."""
    if k == 1:
        return tiny_spheres(n or 20000, 4, seed=1001, shuffle=shuffle), [tiny_camera()]
    if k == 2:
        sc = surfaces_scene(n or 5_000_000, 8, seed=1002, size_scale=SIZE_SCALE_SINGLE_VIEW,
                            shuffle=shuffle)
        return sc, [single_view_camera(seed=1002)]
    if k == 3:
        sc = surfaces_scene(n or 20_000_000, 8, seed=1003, size_scale=SIZE_SCALE_SINGLE_VIEW,
                            shuffle=shuffle)
        return sc, orbit_cameras(16, seed=1003)
    if k == 4:
        sc = surfaces_scene(n or 120_000_000, 4, n_planes=250, n_spheres=250, box=100.0, seed=1004,
                            size_scale=SIZE_SCALE_SINGLE_VIEW, shuffle=shuffle)
        return sc, path_cameras(60, 1920, 1080, seed=1004)
    raise ValueError(k)


# Surface size multiplier of the 10 m-box scenes, chosen once so that the
# single-view 1080p camera sees about 8 distinct surfaces per covered pixel
# (measured 8.2 at 5M points, counting surfaces per covered layer-2 pixel).
SIZE_SCALE_SINGLE_VIEW = 2.5
