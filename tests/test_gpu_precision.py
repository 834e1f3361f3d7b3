"""Error against the FP64 oracle, per output and per descriptor storage type,
at the full single-view size (5M points, 1920x1080, C = 8).

Two errors per output:
* arithmetic: the GPU result against the oracle on the same stored
  descriptors (BF16/FP16 values are exact in FP64), i.e. what FP32 blending
  and accumulation cost;
* storage: the GPU result with BF16/FP16 descriptors against the oracle on
  the FP32 draw they were rounded from, i.e. what storing the descriptors in
  16 bits costs.
Both are printed (run with -s) and bounded: the arithmetic error by the
parity tolerances, the storage error by the 16-bit rounding (2^-9 for BF16,
2^-12 for FP16, relative, propagated through a mean and the gradients).
"""
import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, RTOL_GRAD, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _errs(g, r):
    """max |g - r| / max(|r|, rms(r)) and rms(g - r) / rms(r) per output."""
    out = {}
    for key, gv, rv in (("image", g["img"][0], r["img"][0]), ("dtau", g["dfeat"], r["dfeat"]),
                        ("dx", g["dxyz"], r["dxyz"]), ("dpose", g["dpose"][0], r["dpose"][0]),
                        ("dintr", g["dintr"][0], r["dintr"][0])):
        gv = np.asarray(gv, np.float64)
        rv = np.asarray(rv, np.float64)
        rms = float(np.sqrt(np.mean(rv * rv)))
        den = np.maximum(np.abs(rv), rms)
        den = np.where(den == 0, 1.0, den)
        out[key] = (float(np.max(np.abs(gv - rv) / den)), float(np.sqrt(np.mean((gv - rv) ** 2)) / max(rms, 1e-300)))
    return out


@pytest.fixture(scope="module")
def single_view():
    return scenes.config(2)


def test_error_per_output_and_storage_type(adop, orc, single_view):
    sc, cams = single_view
    G = [scenes.upstream_grad(c.w, c.h, 4, sc.c, 2024) for c in cams]
    ref32 = oracle_run(orc, sc, cams, "f32", grads=G)
    rows = []
    for dtype, unit in (("f32", 2.0 ** -24), ("bf16", 2.0 ** -9), ("f16", 2.0 ** -12)):
        g = gpu_run(adop, sc, cams, dtype, grads=G, grad_assign=True)
        r = ref32 if dtype == "f32" else oracle_run(orc, sc, cams, dtype, grads=G)
        assert all(np.array_equal(a, b) for a, b in zip(g["keys"], r["keys"]))
        arith = _errs(g, r)
        storage = _errs(g, ref32)
        rows.append((dtype, arith, storage))
        assert arith["image"][0] <= RTOL_FEAT_F32
        assert arith["dtau"][0] <= RTOL_GRAD and arith["dx"][0] <= RTOL_GRAD
        # storage: a mean of values each within `unit` relative of the draw
        assert storage["image"][1] <= 4 * unit + 1e-6
    print("\nstorage | output | arithmetic max / rms | storage max / rms")
    for dtype, arith, storage in rows:
        for k in arith:
            print(f"{dtype:5s} | {k:6s} | {arith[k][0]:.2e} / {arith[k][1]:.2e} | {storage[k][0]:.2e} / {storage[k][1]:.2e}")
