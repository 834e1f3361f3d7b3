"""The host-buffer pipeline (paper_2110_06635_gb300.pipeline): steps fed from
pinned host memory, copies overlapping the kernels on three streams and two
alternating device buffer sets.  Each step's results must be those of the
same step run alone through the C ABI, whatever the step before and after
it was, and its inputs must be the ones it was given."""
import numpy as np
import pytest

import scenes
from parity import RTOL_FEAT_F32, RTOL_GRAD, assert_close, gpu_run

pytestmark = pytest.mark.gpu


def test_pipelined_steps_equal_steps_alone(adop):
    import torch
    from paper_2110_06635_gb300.pipeline import HostPipeline, StepIO
    sc0, cams = scenes.config(1)
    cam = cams[0]
    rng = np.random.default_rng(5)
    steps = []
    for k in range(5):  # five different steps: the two buffer sets alternate and are reused
        sc = scenes.Scene(sc0.xyz + rng.normal(scale=2e-3, size=sc0.xyz.shape).astype(np.float32),
                          (sc0.feat * (1.0 + 0.1 * k)).astype(np.float32))
        G = scenes.upstream_grad(cam.w, cam.h, 4, sc.c, 100 + k)
        steps.append((sc, G))
    pipe = HostPipeline(cam, sc0.n, sc0.c, torch.float32, torch.float32, 4)
    ios = []
    for sc, G in steps:
        io = StepIO.alloc(cam, sc.n, sc.c)
        io.xyz.copy_(torch.from_numpy(sc.xyz))
        io.feat.copy_(torch.from_numpy(sc.feat))
        for h, g in zip(io.grads, G):
            h.copy_(torch.from_numpy(np.ascontiguousarray(g, np.float32)))
        ios.append(io)
    pipe.run(ios)
    for (sc, G), io in zip(steps, ios):
        ref = gpu_run(adop, sc, [cam], "f32", grads=[G], grad_assign=True)
        img = np.concatenate([t.numpy().ravel() for t in io.images])
        assert_close(img, ref["img"][0], RTOL_FEAT_F32, "image")
        assert_close(io.grad_feat.numpy(), ref["dfeat"], RTOL_GRAD, "dL/dtau")
        assert_close(io.grad_xyz.numpy(), ref["dxyz"], RTOL_GRAD, "dL/dx")
        assert_close(io.grad_pose.numpy(), ref["dpose"][0], RTOL_GRAD, "dL/dxi")
        assert_close(io.grad_intr.numpy(), ref["dintr"][0], RTOL_GRAD, "dL/dK")
