"""Steps of the forward + backward pass (Sec. 3.1) fed from, and returned to,
pinned host memory, with the copies overlapping the kernels.

A step's inputs (positions, descriptors, upstream gradients of every layer)
are copied host -> device on one CUDA stream, its kernels run on a second
(the C ABI's adop_render_forward / adop_render_backward), and its results
(the image pyramid, dL/dtau, dL/dx, pose and intrinsics gradients) are copied
device -> host on a third.  Two sets of device buffers alternate, so step
k + 1's inputs arrive and step k - 1's results leave while step k computes;
events order each buffer set's reuse.  Every step still moves all of its own
inputs and results across the host link.

All arithmetic is the library's; this module allocates buffers, marshals
pointers and orders streams.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import torch

from . import _abi as A


@dataclass
class StepIO:
    """Pinned host tensors of one step: inputs xyz (n x 3 FP32), feat (n x c),
    grads (one c x h_l x w_l tensor per layer, FP32 or a 16-bit type);
    results images (one c x h_l x w_l tensor per layer, the output dtype),
    grad_feat (n x c, FP32 or a 16-bit type: summed in FP32 on the device and
    rounded once), grad_xyz (n x 3 FP32), grad_pose (6), grad_intr (6)."""
    xyz: torch.Tensor
    feat: torch.Tensor
    grads: list
    images: list
    grad_feat: torch.Tensor
    grad_xyz: torch.Tensor
    grad_pose: torch.Tensor
    grad_intr: torch.Tensor

    @staticmethod
    def alloc(cam, n: int, c: int, feat_dtype=torch.float32, out_dtype=torch.float32, levels: int = 4,
              grad_dtype=torch.float32, grad_feat_dtype=torch.float32):
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True)  # noqa: E731
        w, h = int(cam.w), int(cam.h)
        return StepIO(pin((n, 3), torch.float32), pin((n, c), feat_dtype),
                      [pin((c, h >> l, w >> l), grad_dtype) for l in range(levels)],
                      [pin((c, h >> l, w >> l), out_dtype) for l in range(levels)],
                      pin((n, c), grad_feat_dtype), pin((n, 3), torch.float32), pin((6,), torch.float32),
                      pin((6,), torch.float32))

    def inputs(self):
        return [self.xyz, self.feat, *self.grads]

    def results(self):
        return [*self.images, self.grad_feat, self.grad_xyz, self.grad_pose, self.grad_intr]

    def bytes_in(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.inputs())

    def bytes_out(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.results())


class HostPipeline:
    """Forward + backward of one camera per step from host buffers (see the
    module docstring).  ``flags`` are adop_params flags; gradients of the
    descriptors and positions are assigned (ADOP_FLAG_GRAD_ASSIGN), the pose
    and intrinsics gradients are per step."""

    def __init__(self, cam, n: int, c: int, feat_dtype=torch.float32, out_dtype=torch.float32, levels: int = 4,
                 alpha: float = 0.01, znear: float = 1e-3, flags: int = 0, device="cuda", crf_lut=None,
                 grad_dtype=torch.float32, grad_feat_dtype=torch.float32):
        self.cam, self.n, self.c, self.levels = cam, n, c, levels
        self.device = torch.device(device)
        self.lib = A.load()
        self.params = A.Params(levels, alpha, znear, None, flags | A.ADOP_FLAG_GRAD_ASSIGN)
        self.luts = None if crf_lut is None else [crf_lut]
        w, h = int(cam.w), int(cam.h)
        self.sets = []
        for _ in range(2):
            s = {
                "xyz": torch.empty((n, 3), dtype=torch.float32, device=self.device),
                "feat": torch.empty((n, c), dtype=feat_dtype, device=self.device),
                "grads": [torch.empty((c, h >> l, w >> l), dtype=grad_dtype, device=self.device)
                          for l in range(levels)],
                "frame": A.Frame.alloc(cam, c, levels, out_dtype, True, self.device, n),
                "gfeat": torch.empty((n, c), dtype=grad_feat_dtype, device=self.device),
                "gxyz": torch.empty((n, 3), dtype=torch.float32, device=self.device),
                "gpose": torch.zeros((1, 6), dtype=torch.float32, device=self.device),
                "gintr": torch.zeros((1, 6), dtype=torch.float32, device=self.device),
            }
            pts = A.Points(s["xyz"], s["feat"])
            s["ps"] = pts.struct()
            s["fr"] = (A.adop_frame * 1)(s["frame"].struct())
            s["g"] = (ct.c_void_p * levels)(*[g.data_ptr() for g in s["grads"]])
            self.sets.append(s)
        self.ws = A.alloc_workspace(A.Points(self.sets[0]["xyz"], self.sets[0]["feat"]), [cam], self.params,
                                    self.luts, self.device)
        self.wp, self.wn = A._ws_ptr(self.ws)
        self.pr = self.params.struct()
        self.pr.grad_dtype = A.dtype_code(grad_dtype)
        self.pr.grad_feat_dtype = A.dtype_code(grad_feat_dtype)
        self.cams = A._cams_array([cam], self.luts)
        self.s_in, self.s_comp, self.s_out = (torch.cuda.Stream(self.device) for _ in range(3))

    def _compute(self, s, stream):
        sp = ct.c_void_p(stream.cuda_stream)
        st = self.lib.adop_render_forward(ct.byref(s["ps"]), self.cams, 1, ct.byref(self.pr), s["fr"], self.wp,
                                          self.wn, sp)
        if st != 0:
            raise A.AdopError(st, self.lib.adop_last_error().decode())
        st = self.lib.adop_render_backward(ct.byref(s["ps"]), self.cams, 1, ct.byref(self.pr), s["fr"], s["g"],
                                           s["gfeat"].data_ptr(), s["gxyz"].data_ptr(), s["gpose"].data_ptr(),
                                           s["gintr"].data_ptr(), self.wp, self.wn, sp)
        if st != 0:
            raise A.AdopError(st, self.lib.adop_last_error().decode())

    def run(self, steps, start=None, end=None):
        """Run every StepIO in `steps` in order; returns when all results are
        in host memory.  `start` (a recorded CUDA event) gates the first
        copy; `end` is recorded after the last one (for timing)."""
        ev_in = [torch.cuda.Event() for _ in range(2)]    # inputs of the set copied in
        ev_comp = [torch.cuda.Event() for _ in range(2)]  # the set's kernels done (inputs free)
        ev_out = [torch.cuda.Event() for _ in range(2)]   # the set's results copied out
        used = [False, False]
        if start is not None:
            self.s_in.wait_event(start)
        for k, io in enumerate(steps):
            b = k & 1
            s = self.sets[b]
            with torch.cuda.stream(self.s_in):
                if used[b]:
                    self.s_in.wait_event(ev_comp[b])
                for d, h in zip([s["xyz"], s["feat"], *s["grads"]], io.inputs()):
                    d.copy_(h, non_blocking=True)
                ev_in[b].record(self.s_in)
            with torch.cuda.stream(self.s_comp):
                self.s_comp.wait_event(ev_in[b])
                if used[b]:
                    self.s_comp.wait_event(ev_out[b])
                s["gpose"].zero_()
                s["gintr"].zero_()
                self._compute(s, self.s_comp)
                ev_comp[b].record(self.s_comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(ev_comp[b])
                res = [*s["frame"].images, s["gfeat"], s["gxyz"], s["gpose"].view(6), s["gintr"].view(6)]
                for h, d in zip(io.results(), res):
                    h.copy_(d, non_blocking=True)
                ev_out[b].record(self.s_out)
            used[b] = True
        if end is not None:
            end.record(self.s_out)
        self.s_out.synchronize()
