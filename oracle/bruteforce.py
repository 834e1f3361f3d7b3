"""List-based brute-force statement of Eq. blend and Eq. spatialderiv (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Pure-Python loops for tiny
scenes (tens of points, a few hundred pixels): for every pixel it scans every
point, builds the point list Lambda explicitly and evaluates the paper's
formulas literally on the lists -- the representation the paper's three-pass
renderer avoids storing.  It takes the projected pixels and FP32 depths of
each point as input (the projection is pinned separately), so it checks the
depth test, blending and the induced-change rule of ``adop_oracle.c``
independently of how that file organises them.

``shift_rerender`` moves one point's pixel for real and re-evaluates the
target pixel from its list: the exact change that Eq. spatialderiv
approximates.
"""
from __future__ import annotations

import math

import numpy as np


def _f32(x) -> np.float32:
    return np.float32(x)


def _lists(pix, l, p, n):
    return [i for i in range(n) if pix[i][l] == p]


def bruteforce_render(pix, z, feat, w, h, levels, alpha=0.01, background=None):
    """Per layer: min depth, key, Lambda list, |Lambda| and the mean image.

    pix   n x levels pixel ids (-1 = discarded); z  n float32 depths;
    feat  n x c float64.  Returns a list over layers of dicts with per-pixel
    lists ``lam``, ``minz`` (float32 or None), ``key`` (int or None),
    ``I`` (c x h_l x w_l)."""
    n, c = feat.shape
    a1 = _f32(_f32(1.0) + _f32(alpha))
    bg = np.zeros(c) if background is None else np.asarray(background, dtype=np.float64)
    out = []
    for l in range(levels):
        wl, hl = w >> l, h >> l
        lam, minz, key = [], [], []
        I = np.zeros((c, hl, wl))
        for p in range(wl * hl):
            hit = _lists(pix, l, p, n)
            if not hit:
                lam.append([])
                minz.append(None)
                key.append(None)
                I[:, p // wl, p % wl] = bg
                continue
            zmin = min(_f32(z[i]) for i in hit)
            imin = min(i for i in hit if _f32(z[i]) == zmin)
            thr = _f32(zmin * a1)
            members = [i for i in hit if _f32(z[i]) <= thr]
            lam.append(members)
            minz.append(zmin)
            key.append((int(np.float32(zmin).view(np.uint32)) << 32) | imin)
            for ch in range(c):
                I[ch, p // wl, p % wl] = math.fsum(feat[i, ch] for i in members) / len(members)
        out.append({"lam": lam, "minz": minz, "key": key, "I": I, "w": wl, "h": hl})
    return out


def induced_change(layer, i, zi, tau, q, alpha=0.01):
    """Eq. spatialderiv at target pixel q for point i (depth zi, feature tau),
    using the target's explicit list.  Returns (case, Delta I)."""
    a1 = _f32(_f32(1.0) + _f32(alpha))
    wl = layer["w"]
    Iq = layer["I"][:, q // wl, q % wl]
    lam_q = layer["lam"][q]
    if not lam_q:
        return 1, tau - Iq
    mz = layer["minz"][q]
    if _f32(zi) > _f32(mz * a1):
        return 2, np.zeros_like(tau)
    if _f32(_f32(zi) * a1) < mz:
        return 3, tau - Iq
    k = len(lam_q)
    return 4, (k * Iq + tau) / (1 + k) - Iq


def bruteforce_spatial(pix, z, feat, G_layers, w, h, levels, alpha=0.01, background=None,
                       all_projected=False):
    """g_u, g_v (layer pixel units) of every point at every layer, plus dL/dtau,
    from the explicit lists (Eqs. induce, gradp, spatialderiv)."""
    n, c = feat.shape
    layers = bruteforce_render(pix, z, feat, w, h, levels, alpha, background)
    gu = np.zeros((n, levels))
    gv = np.zeros((n, levels))
    dfeat = np.zeros((n, c))
    for l, L in enumerate(layers):
        wl, hl = L["w"], L["h"]
        Gl = G_layers[l]
        for i in range(n):
            p = pix[i][l]
            if p < 0:
                continue
            member = i in L["lam"][p]
            if member:
                dfeat[i] += Gl[:, p // wl, p % wl] / len(L["lam"][p])
            if not member and not all_projected:
                continue
            pu, pv = p % wl, p // wl

            def contrib(qu, qv):
                if not (0 <= qu < wl and 0 <= qv < hl):
                    return 0.0
                q = qv * wl + qu
                _, d = induced_change(L, i, z[i], feat[i], q, alpha)
                return float(np.dot(Gl[:, qv, qu], d))

            gu[i, l] = 0.5 * (contrib(pu + 1, pv) - contrib(pu - 1, pv))
            gv[i, l] = 0.5 * (contrib(pu, pv + 1) - contrib(pu, pv - 1))
    return layers, dfeat, gu, gv


def shift_rerender(pix, z, feat, w, h, levels, l, i, q, alpha=0.01, background=None):
    """Move point i's layer-l pixel to q for real, re-render q from its list
    and return I'(q) - I(q): the exact change at the target pixel."""
    moved = [list(r) for r in pix]
    moved[i][l] = q
    return (_render_pixel(moved, z, feat, l, q, alpha, background)
            - _render_pixel(pix, z, feat, l, q, alpha, background))


def _render_pixel(pix, z, feat, l, p, alpha, background):
    """Eq. depthtest + Eq. blend for a single pixel from its explicit list."""
    n, c = feat.shape
    a1 = _f32(_f32(1.0) + _f32(alpha))
    hit = _lists(pix, l, p, n)
    if not hit:
        return np.zeros(c) if background is None else np.asarray(background, dtype=np.float64)
    thr = _f32(min(_f32(z[i]) for i in hit) * a1)
    members = [i for i in hit if _f32(z[i]) <= thr]
    return np.array([math.fsum(feat[i, ch] for i in members) / len(members) for ch in range(c)])
