"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every symbol that include/adop.h declares, and argument errors
are reported synchronously, before any CUDA call."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2110_06635_gb300 as adop
    adop.build()
    return adop, adop.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(adop_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    adop, so = lib
    names = declared_functions()
    assert "adop_render_forward" in names and "adop_render_backward" in names
    for name in names:
        assert hasattr(so, name), f"{name} declared in include/ but not exported"
    assert set(names) <= set(adop.SIGNATURES), "binding misses a declared entry point"
    assert adop.adop_abi_version() == 3


def _structs(adop, n=10, c=4, levels=4, w=64, h=48, flags=0):
    from paper_2110_06635_gb300 import _abi as A
    pts = A.adop_points(n, c, A.ADOP_F32, 0x10000, 0x20000, None)
    K = A.adop_intrinsics(w, h, 50.0, 50.0, w / 2, h / 2, 0, 0, 0, 0, 0, 0)
    R = (ct.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    T = A.adop_pose(R, (ct.c_float * 3)(0, 0, 2))
    cam = (A.adop_camera * 1)(A.adop_camera(K, T, A.adop_photometric()))
    prm = A.adop_params(levels, 0.01, 1e-3, None, flags)
    fr = (A.adop_frame * 1)()
    return pts, cam, prm, fr


def _fwd(so, pts, cam, prm, fr, ws=0x100000, nbytes=1 << 40, ncam=1):
    return so.adop_render_forward(ct.byref(pts), cam, ncam, ct.byref(prm), fr, ws, nbytes, None)


def test_workspace_bytes(lib):
    adop, so = lib
    pts, cam, prm, fr = _structs(adop)
    n = so.adop_workspace_bytes(ct.byref(pts), cam, 1, ct.byref(prm))
    px = 64 * 48 + 32 * 24 + 16 * 12 + 8 * 6
    assert n >= px * (8 + 4 + 16 + 32) and n % 256 == 0
    prm.levels = 0
    assert so.adop_workspace_bytes(ct.byref(pts), cam, 1, ct.byref(prm)) == 0
    assert "levels" in so.adop_last_error().decode()


@pytest.mark.parametrize("case,status,msg", [
    ("ncam0", 1, "n_cam"), ("levels9", 1, "levels"), ("c5", 2, "channel count 5"), ("alpha", 1, "alpha"),
    ("znear", 1, "znear"), ("flags", 1, "flag"), ("cull", 1, "normals"), ("size", 1, "image size"),
    ("small", 1, "too small"), ("ws", 3, "workspace"), ("wsalign", 1, "aligned"), ("feat", 1, "16-byte"),
    ("mixed", 1, "all set or all NULL"), ("nan", 1, "non-finite"), ("dtype", 1, "dtype"),
    ("envsize", 1, "environment map"), ("envalign", 1, "env must be 16-byte aligned"),
])
def test_invalid_arguments_fail_synchronously(lib, case, status, msg):
    adop, so = lib
    pts, cam, prm, fr = _structs(adop)
    kw = {}
    if case == "ncam0":
        kw["ncam"] = 0
    elif case == "levels9":
        prm.levels = 9
    elif case == "c5":
        pts.c = 5
    elif case == "alpha":
        prm.alpha = -1.0
    elif case == "znear":
        prm.znear = float("nan")
    elif case == "flags":
        prm.flags = 1 << 12
    elif case == "cull":
        prm.flags = adop.ADOP_FLAG_NORMAL_CULL
    elif case == "size":
        cam[0].K.w = 0
    elif case == "small":
        cam[0].K.w = 4
    elif case == "ws":
        kw["nbytes"] = 1024
    elif case == "wsalign":
        kw["ws"] = 0x100010
    elif case == "feat":
        pts.feat = 0x20008
    elif case == "mixed":
        fr[0].key[0] = 0x40000
    elif case == "nan":
        cam[0].T.t[1] = float("inf")
    elif case == "dtype":
        fr[0].out_dtype = 7
    elif case == "envsize":
        prm.env, prm.env_w, prm.env_h = 0x50000, 64, 0
    elif case == "envalign":
        prm.env, prm.env_w, prm.env_h = 0x50008, 64, 32
    st = _fwd(so, pts, cam, prm, fr, **kw)
    assert st == status
    assert msg in so.adop_last_error().decode()


def test_backward_validates_too(lib):
    adop, so = lib
    pts, cam, prm, fr = _structs(adop)
    prm.levels = 12
    st = so.adop_render_backward(ct.byref(pts), cam, 1, ct.byref(prm), fr, None, None, None, None, None,
                                 0x100000, 1 << 40, None)
    assert st == 1 and "levels" in so.adop_last_error().decode()


def test_env_backward_validates(lib):
    adop, so = lib
    pts, cam, prm, fr = _structs(adop)
    g = ct.c_void_p(0x60000)
    # no environment map in the params
    st = so.adop_env_backward(cam, 1, ct.byref(prm), 8, fr, None, g, None)
    assert st == 1 and "env" in so.adop_last_error().decode()
    prm.env, prm.env_w, prm.env_h = 0x50000, 20000, 16
    st = so.adop_env_backward(cam, 1, ct.byref(prm), 8, fr, None, g, None)
    assert st == 1 and "16384" in so.adop_last_error().decode()
    prm.env_w = 64
    st = so.adop_env_backward(cam, 1, ct.byref(prm), 5, fr, None, g, None)
    assert st == 2
    # frames without the forward's counts
    st = so.adop_env_backward(cam, 1, ct.byref(prm), 8, fr, None, g, None)
    assert st == 1 and "count" in so.adop_last_error().decode()


@pytest.mark.parametrize("entry", ["adop_render_backward", "adop_render_backward_noalloc"])
def test_grad_images_checked_before_launch(lib, entry):
    """Both backward wrappers read every upstream gradient as c x h_l x w_l
    values of one floating type (float32, bfloat16 or float16): another
    dtype, mixed dtypes or another size is refused on the host (the tensors
    here are CPU tensors, so nothing could have been launched)."""
    import numpy as np
    import torch
    import scenes
    adop, _ = lib
    cam = scenes.Camera(64, 48, 50.0, 50.0, 32.0, 24.0, R=np.eye(3, dtype=np.float32),
                        t=np.array([0, 0, 2], np.float32))
    pts = adop.Points(torch.zeros((10, 3)), torch.zeros((10, 4)))
    params = adop.Params(2, 0.01, 1e-3, None, 0)
    fn = getattr(adop, entry)
    extra = [None] * 4 + ([torch.zeros(1)] if entry == "adop_render_backward" else [])
    bad_dtype = [[torch.zeros((4, 48, 64), dtype=torch.int32), None]]
    with pytest.raises(ValueError, match="float32"):
        fn(pts, [cam], params, [None], bad_dtype, *extra)
    mixed = [[torch.zeros((4, 48, 64), dtype=torch.bfloat16), torch.zeros((4, 24, 32))]]
    with pytest.raises(ValueError, match="mix"):
        fn(pts, [cam], params, [None], mixed, *extra)
    bad_size = [[None, torch.zeros((4, 24, 31))]]
    with pytest.raises(ValueError, match="elements"):
        fn(pts, [cam], params, [None], bad_size, *extra)


def test_gradient_dtype_rules(lib):
    """The backward's storage types are checked before any launch: a 16-bit
    grad_feat only when gradients are assigned for one camera; an unknown
    dtype code is an argument error."""
    adop, so = lib
    from paper_2110_06635_gb300 import _abi as A
    pts, cam, prm, fr = _structs(adop)
    for k in range(4):
        fr[0].key[k] = 0x300000
        fr[0].count[k] = 0x400000
    fr[0].acc = 0x500000
    g = (ct.c_void_p * 4)()
    call = lambda: so.adop_render_backward(ct.byref(pts), cam, 1, ct.byref(prm), fr, g, 0x600000, None, None, None,
                                           0x100000, 1 << 40, None)
    prm.grad_feat_dtype = A.ADOP_BF16
    assert call() == 2 and "ADOP_FLAG_GRAD_ASSIGN" in adop.adop_last_error()
    prm.grad_feat_dtype = 7
    assert call() == 1 and "dtype" in adop.adop_last_error()
    prm.grad_feat_dtype = A.ADOP_F32
    prm.grad_dtype = 9
    assert call() == 1 and "dtype" in adop.adop_last_error()


def test_server_config_refused_before_any_cuda_call(lib):
    """adop_serve_create checks its configuration on the host and allocates
    nothing for a bad one: the batching window, batch size, stream and slot
    counts."""
    adop, so = lib
    from paper_2110_06635_gb300 import _abi as A
    good = dict(mem_budget_bytes=64 << 20, max_slots=8, streams=2, max_batch=4, levels=4, alpha=0.01, znear=1e-3,
                flags=0, out_dtype=A.ADOP_F32, background=None, env=None, env_w=0, env_h=0, batch_window_us=0)
    for field, bad, msg in (("batch_window_us", -1, "batch_window_us"), ("batch_window_us", 2_000_000, "batch_window_us"),
                            ("max_batch", 0, "max_batch"), ("max_batch", 17, "max_batch"), ("streams", 0, "streams"),
                            ("max_slots", 0, "max_slots"), ("mem_budget_bytes", 1024, "budget"),
                            ("flags", A.ADOP_FLAG_DISCARD, "flags")):
        cfg = A.adop_serve_config(**{**good, field: bad})
        h = ct.c_void_p()
        assert so.adop_serve_create(ct.byref(cfg), ct.byref(h)) == 1, field
        assert msg in adop.adop_last_error(), (field, adop.adop_last_error())
        assert not h.value
