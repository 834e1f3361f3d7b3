"""The differentiable render frees a step's frames and workspace as soon as
its outputs are dropped: nothing in the autograd context refers back to the
outputs (no reference cycle for Python's cycle collector to find later).
The library calls are replaced by stand-ins, so this runs on the CPU."""
import gc
import weakref

import pytest
import torch

import scenes
from paper_2110_06635_gb300 import _abi as A
from paper_2110_06635_gb300 import autograd as AG


@pytest.fixture
def stubbed(monkeypatch):
    rec = {"ws": [], "bwd_frames": None}

    def alloc_workspace(points, cams, params, crf_luts=None, device="cuda"):
        t = torch.empty(4096, dtype=torch.uint8, device=device)
        rec["ws"].append(weakref.ref(t))
        return t

    def render_forward(pts, cams, params, frames, ws, crf_luts=None):
        for f in frames:
            for im in f.images:
                im.zero_()

    def render_backward(pts, cams, params, frames, gimgs, gfeat, gxyz, gpose, gintr, ws, crf_luts=None):
        rec["bwd_frames"] = [(f.key is not None, f.count is not None, f.acc is not None, len(f.images))
                             for f in frames]
        for g in (gfeat, gxyz, gpose, gintr):
            if g is not None:
                g.zero_()

    monkeypatch.setattr(A, "alloc_workspace", alloc_workspace)
    monkeypatch.setattr(A, "adop_render_forward", render_forward)
    monkeypatch.setattr(A, "adop_render_backward", render_backward)
    return rec


def _inputs():
    cam = scenes.Camera(64, 48, 50.0, 50.0, 32.0, 24.0)
    xyz = torch.zeros(10, 3, requires_grad=True)
    feat = torch.zeros(10, 4, requires_grad=True)
    return [cam, cam], xyz, feat


@pytest.mark.parametrize("keep_state", [True, False])
def test_step_freed_with_its_outputs(stubbed, keep_state):
    cams, xyz, feat = _inputs()
    was = gc.isenabled()
    gc.disable()
    try:
        out = AG.rasterize(xyz, feat, cams, levels=2, keep_state=keep_state)
        loss = sum(im.sum() for row in out for im in row)
        loss.backward()
        # the backward gets each frame's per-pixel state (when kept), without its images
        assert stubbed["bwd_frames"] == [(keep_state, keep_state, keep_state, 0)] * 2
        assert stubbed["ws"][0]() is not None  # still referenced by the graph
        del out, loss
        assert stubbed["ws"][0]() is None, "workspace outlived the step's outputs"
    finally:
        if was:
            gc.enable()


def test_forward_only_step_freed(stubbed):
    cams, xyz, feat = _inputs()
    was = gc.isenabled()
    gc.disable()
    try:
        out = AG.rasterize(xyz, feat, cams, levels=2)
        images = [im for row in out for im in row]
        assert all(im.grad_fn is not None for im in images)
        del out, images
        assert stubbed["ws"][0]() is None, "workspace outlived the step's outputs"
    finally:
        if was:
            gc.enable()
