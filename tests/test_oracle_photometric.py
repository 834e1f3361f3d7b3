"""Pins of the oracle's photometric camera model (Sec. 3.3: exposure, white
balance, vignette, response curve; Eq. resonseleak for the training response)
and of its parameter gradients.  CPU only."""
import numpy as np
import pytest


def test_closed_form_single_pixels(orc):
    # identity response: out = I * 2^-EV * wb * (1 + a2 r^2 + a4 r^4 + a6 r^6)
    img = np.ones((3, 2, 2))
    out = orc.epilogue(img, ev=1.0, wb=(2.0, 1.0, 0.5), vig_c=(0.5, 0.5), vig_a=(-0.1, 0.2, 0.05))
    # pixel (u=0, v=0): r^2 = 0.5, vignette = 1 - 0.05 + 0.05 + 0.00625 = 1.00625
    assert np.isclose(out[0, 0, 0], 0.5 * 2.0 * 1.00625, rtol=0, atol=1e-15)
    assert np.isclose(out[2, 0, 0], 0.5 * 0.5 * 1.00625, rtol=0, atol=1e-15)
    # pixel (u=1, v=1): (0.5, 0.5) - c_v = 0: no vignette
    assert np.isclose(out[1, 1, 1], 0.5, rtol=0, atol=1e-15)


def test_lut_knots_clamp_and_leak(orc):
    n = 11
    lut = np.stack([np.linspace(0, 1, n) ** 0.45] * 3)
    # at a knot the interpolation returns the sample itself; outside [0,1] it clamps
    img = np.array([[[0.3, 1.7, -0.4]]] * 3)
    out = orc.epilogue(img, crf=lut)
    assert np.isclose(out[0, 0, 0], lut[0, 3], rtol=0, atol=1e-15)
    assert out[0, 0, 1] == lut[0, -1] and out[0, 0, 2] == lut[0, 0]
    # Eq. resonseleak, alpha = 0.01: 0.01 x below 0, -0.01/sqrt(x) + 1.01 above 1
    img = np.array([[[4.0, -2.0, 0.3]]] * 3)
    out = orc.epilogue(img, crf=lut, leaky=True)
    assert np.isclose(out[0, 0, 0], -0.01 / 2.0 + 1.01, rtol=0, atol=1e-15)
    assert np.isclose(out[0, 0, 1], -0.02, rtol=0, atol=1e-15)
    assert np.isclose(out[0, 0, 2], lut[0, 3], rtol=0, atol=1e-15)
    # the leaky curve is continuous at 1 when R(1) = 1 and bounded by 1.01
    assert np.isclose(orc.epilogue(np.full((3, 1, 1), 1.0 + 1e-12), crf=lut, leaky=True)[0, 0, 0], 1.0)
    assert orc.epilogue(np.full((3, 1, 1), 1e12), crf=lut, leaky=True)[0, 0, 0] < 1.01


def _params(rng):
    return dict(ev=float(rng.uniform(-1, 1)), wb=tuple(rng.uniform(0.8, 1.2, 3)), vig_c=tuple(rng.uniform(0.4, 0.6, 2)),
                vig_a=tuple(rng.uniform(-0.2, 0.2, 3)))


@pytest.mark.parametrize("leaky", [False, True])
def test_parameter_gradients_match_finite_differences(orc, leaky):
    rng = np.random.default_rng(3 + leaky)
    c, h, w = 4, 9, 13
    img = rng.uniform(-0.3, 1.6, size=(c, h, w))
    G = rng.normal(size=(c, h, w))
    lut = np.stack([np.sort(rng.random(17)) for _ in range(3)])
    lut[:, 0], lut[:, -1] = 0.0, 1.0
    p = _params(rng)
    gp, gcrf = orc.photometric_grad(img, G, crf=lut, leaky=leaky, **p)

    def L(**q):
        kw = dict(p)
        kw.update(q)
        return float(np.sum(G * orc.epilogue(img, crf=kw.pop("crf", lut), leaky=leaky, **kw)))

    eps = 1e-7
    fd = [(L(ev=p["ev"] + eps) - L(ev=p["ev"] - eps)) / (2 * eps)]
    for ch in range(3):
        wp, wm = list(p["wb"]), list(p["wb"])
        wp[ch] += eps
        wm[ch] -= eps
        fd.append((L(wb=tuple(wp)) - L(wb=tuple(wm))) / (2 * eps))
    for k in range(2):
        cp, cm = list(p["vig_c"]), list(p["vig_c"])
        cp[k] += eps
        cm[k] -= eps
        fd.append((L(vig_c=tuple(cp)) - L(vig_c=tuple(cm))) / (2 * eps))
    for k in range(3):
        ap, am = list(p["vig_a"]), list(p["vig_a"])
        ap[k] += eps
        am[k] -= eps
        fd.append((L(vig_a=tuple(ap)) - L(vig_a=tuple(am))) / (2 * eps))
    assert np.allclose(gp, fd, rtol=1e-5, atol=1e-6), (gp, fd)
    # the response curve is linear in its samples: any step is exact
    for ch, j in [(0, 0), (1, 7), (2, 16), (0, 9)]:
        lp = lut.copy()
        lp[ch, j] += 1.0
        assert np.isclose(L(crf=lp) - L(), gcrf[ch, j], rtol=1e-9, atol=1e-9)
    # and the chained d out / d I against finite differences of the input
    _, dI = orc.epilogue(img, crf=lut, leaky=leaky, want_grad=True, **p)
    for (ch, v, u) in [(0, 1, 2), (2, 5, 7), (1, 8, 12), (3, 0, 0)]:
        ip, im = img.copy(), img.copy()
        ip[ch, v, u] += eps
        im[ch, v, u] -= eps
        fdI = (orc.epilogue(ip, crf=lut, leaky=leaky, **p)[ch, v, u] - orc.epilogue(im, crf=lut, leaky=leaky, **p)[ch, v, u]) / (2 * eps)
        assert np.isclose(dI[ch, v, u], fdI, rtol=1e-5, atol=1e-7)
