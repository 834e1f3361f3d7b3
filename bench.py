#!/usr/bin/env python
"""Throughput of ADOP's differentiable one-pixel point rasterizer (forward +
backward) on one camera view at 1920x1080.

Workload (default): 5,000,000 points on 25 planes and 25 spheres in a 10 m box
(depth complexity ~8), 8 descriptor channels stored in BF16 (FP32 measured
beside it), a distorted pinhole camera (fx = fy = 1500, k1 = -0.05, k2 = 0.01)
12 m from the centre, 4 pyramid layers, fuzzy threshold alpha = 0.01; forward
plus backward to descriptors, positions, the 6-DoF pose and intrinsics.  One
step = one forward + one backward of that view through the C ABI.

Metric: points/s (points processed through all 4 layers of one camera,
forward + backward) -- higher is better.  The JSON line also carries the
roofline of the dominant kernel, the FP32 comparison, an end-to-end number
with host buffers, the clock record and the CPU oracle's rate.

--impl reference times the CPU oracle (the plain FP64 statement of the
method) on the same workload, a bounded sample of points per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "points/sec fwd+bwd at 1920x1080 (BF16 vs FP32, % HBM roofline); served p50/p99 ms"
UNIT = "points/s"
L2_FLUSH_BYTES = 256 << 20
LEVELS = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--points", type=int, default=5_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="a few steps, no extras (for ncu)")
    ap.add_argument("--profile-large", action="store_true",
                    help="only the 120M-point forward + backward in BF16, a few steps (for an ncu launch list)")
    ap.add_argument("--no-train", action="store_true", help="skip the 16-camera training step")
    ap.add_argument("--no-discard", action="store_true", help="skip the stochastic-discarding variant")
    ap.add_argument("--no-env", action="store_true", help="skip the environment-map variant")
    ap.add_argument("--no-shuffle", action="store_true", help="skip the randomly ordered variant")
    ap.add_argument("--eager", action="store_true", help="time the step launched eagerly, not as a CUDA graph")
    ap.add_argument("--no-large", action="store_true", help="skip the 120M-point large scene")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--record-traffic", nargs="+", metavar="NCU_CSV",
                    help="write profiles/ncu_traffic.json from ncu --csv logs of single-kernel captures "
                         "(DRAM bytes and L2 atomic requests per launch) and exit")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas, no data exchange)
# ---------------------------------------------------------------------------

def dist_setup(backend=None):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    if backend is None:
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return dist, dist.get_rank(), dist.get_world_size()


def max_over_ranks(dist, value: float, device) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(step, k: int, flush=None, dist=None, device="cuda"):
    """Time exactly k calls of step(): barrier + synchronize on both sides,
    per-step CUDA events on the current stream (an optional L2 flush between
    steps is outside the events).  Returns (total device ms, per-step ms)."""
    import torch
    cuda = str(device).startswith("cuda")
    if dist is not None:
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()
    times = []
    if cuda:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            if flush is not None:
                flush()
            evs[i][0].record()
            step()
            evs[i][1].record()
        torch.cuda.synchronize()
        times = [a.elapsed_time(b) for a, b in evs]
    else:
        for i in range(k):
            if flush is not None:
                flush()
            t0 = time.perf_counter()
            step()
            times.append((time.perf_counter() - t0) * 1e3)
    if dist is not None:
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()
    return float(sum(times)), times


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes; no
    package needed): one GPU's SM clock, its maximum and the clock-event
    reason mask.  Nothing is set.  Raises OSError where NVML is missing."""
    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL = 0x4, 0x8, 0x20, 0x40
    CLOCK_SM = 1

    def __init__(self, uuid: str):
        import ctypes as ct
        self.ct = ct
        self.lib = ct.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.dev = ct.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ct.byref(self.dev)) != 0:
            self.lib.nvmlShutdown()
            raise OSError(f"no NVML device {uuid}")
        self.reasons_fn = (getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or
                           self.lib.nvmlDeviceGetCurrentClocksThrottleReasons)

    def sample(self):
        """(SM MHz, max SM MHz, reason mask), or None if a query failed."""
        ct = self.ct
        c, m, r = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.dev, self.CLOCK_SM, ct.byref(c)) != 0 or
                self.lib.nvmlDeviceGetMaxClockInfo(self.dev, self.CLOCK_SM, ct.byref(m)) != 0 or
                self.reasons_fn(self.dev, ct.byref(r)) != 0):
            return None
        return c.value, m.value, r.value

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """Clocks and throttle reasons during a timed region: `nvidia-smi -lms 200`
    (started, and its first line awaited, before the region) plus NVML polled
    every 1 ms from a thread, so that a region of a few milliseconds still
    gets samples.  Only the samples taken inside the `with` body count."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str, poll_s: float = 0.001):
        self.gpu_id = gpu_id
        self.poll_s = poll_s
        self.proc = None
        self.lines = []
        self.nvml_samples = []
        self.nvml = None
        self.error = ""
        self.stop = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError) as e:
            self.proc = None
            self.error = repr(e)
        try:
            self.nvml = Nvml(self.gpu_id)
            self.poller = threading.Thread(target=self._poll, daemon=True)
            self.poller.start()
        except (OSError, AttributeError) as e:
            self.nvml = None
            self.error = (self.error + " " + repr(e)).strip()
        t0 = time.time()
        while self.proc is not None and not self.lines and self.proc.poll() is None and time.time() - t0 < 3.0:
            time.sleep(0.01)
        self.lines.clear()  # (the region starts here)
        self.nvml_samples.clear()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def _poll(self):
        while not self.stop.is_set():
            v = self.nvml.sample()
            if v is not None:
                self.nvml_samples.append(v)
            time.sleep(self.poll_s)

    def __exit__(self, *exc):
        n_lines = len(self.lines)
        self.stop.set()
        if self.nvml is not None:
            self.poller.join(timeout=2)
            self.nvml.close()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)
        del self.lines[n_lines:]  # lines printed after the region do not count

    def summary(self):
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(self.REASONS, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        n_smi = len(sm)
        bits = dict(zip(self.REASONS, (Nvml.HW_SLOWDOWN, Nvml.HW_THERMAL, Nvml.SW_THERMAL, Nvml.SW_POWER_CAP)))
        for c, m, r in self.nvml_samples:
            sm.append(float(c))
            smax.append(float(m))
            for nm, b in bits.items():
                if r & b:
                    reasons.add(nm)
        if not sm:
            why = self.error or (self.lines[0][:160] if self.lines else "no output")
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, "error": why}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "samples_nvidia_smi": n_smi, "samples_nvml": len(self.nvml_samples)}


def gpu_index(device) -> str:
    """nvidia-smi id of a torch device: its UUID (robust to CUDA_VISIBLE_DEVICES)."""
    import torch
    u = str(torch.cuda.get_device_properties(device).uuid)
    return u if u.startswith("GPU-") else f"GPU-{u}"


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/ncu_traffic.json), or None if the kernel's sources changed
    since the capture (source hash mismatch) or none was recorded."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d:
        return None
    h = hashlib.sha1()
    for rel in d["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return d["dram_bytes_per_launch"] if h.hexdigest() == d["sources_sha1"] else None


def recorded_atomics(kernel: str):
    """L2 atomic requests per launch and the L2 atomic unit's busy fraction
    for `kernel` from the same ncu summary, or None (as recorded_traffic)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d or "l2_atomic_requests_per_launch" not in d:
        return None
    h = hashlib.sha1()
    for rel in d["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != d["sources_sha1"]:
        return None
    return d["l2_atomic_requests_per_launch"], d.get("l2_atomic_unit_active_pct")


# bench name of each library kernel (the k_bin_* launches are one entry)
NCU_KERNELS = {"k_clear": "clear", "k_depth": "depth", "k_accum": "accumulate", "k_normalize": "normalize",
               "k_bwd_prepass": "bwd_prepass", "k_bin_count_blk": "bwd_bin", "k_bin_scan": "bwd_bin",
               "k_bin_scatter_blk": "bwd_bin", "k_bwd_items": "bwd_points", "k_bwd_reduce": "bwd_reduce"}
NCU_SOURCES = {"forward": ["paper_2110_06635_gb300/csrc/forward.cu", "paper_2110_06635_gb300/csrc/adop_device.cuh"],
               "backward": ["paper_2110_06635_gb300/csrc/backward.cu", "paper_2110_06635_gb300/csrc/adop_device.cuh"]}


def record_traffic(csv_paths) -> dict:
    """profiles/ncu_traffic.json from ncu --csv logs (metrics
    gpu__time_duration.sum, dram__bytes_read.sum, dram__bytes_write.sum,
    lts__t_requests_op_atom.sum, lts__t_requests_op_red.sum and
    lts__d_atomic_input_cycles_active.avg.pct_of_peak_sustained_elapsed),
    each capturing launches of one kernel: per bench kernel name, the mean
    per launch, with the SHA-1 of the sources it was taken from (bench.py
    reports a record only while the hash matches)."""
    import csv
    import hashlib
    launches = {}  # (bench name, ncu kernel, launch id) -> {metric: value}
    for path in csv_paths:
        with open(path) as f:
            rows = [r for r in csv.reader(f) if r]
        head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
        cols = rows[head]
        ki, mi, vi, ii = (cols.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "ID"))
        for r in rows[head + 1:]:
            if len(r) <= vi:
                continue
            base = r[ki].split("(")[0].split("<")[0].split("::")[-1].replace("void ", "").strip()
            name = NCU_KERNELS.get(base)
            if name is None:
                continue
            launches.setdefault((name, r[ki].split("(")[0].replace("void ", "").replace("adop::", "").strip(), r[ii]),
                                {})[r[mi]] = float(r[vi].replace(",", ""))
    out = {}
    for name in sorted(set(k[0] for k in launches)):
        per_kernel = {}
        for (nm, kern, _), m in launches.items():
            if nm == name:
                per_kernel.setdefault(kern, []).append(m)
        # a bench entry made of several kernels (binning) sums their per-launch means
        dram = sum(np.mean([x.get("dram__bytes_read.sum", 0) + x.get("dram__bytes_write.sum", 0) for x in v])
                   for v in per_kernel.values())
        atom = sum(np.mean([x.get("lts__t_requests_op_atom.sum", 0) + x.get("lts__t_requests_op_red.sum", 0)
                            for x in v]) for v in per_kernel.values())
        dur = sum(np.mean([x.get("gpu__time_duration.sum", 0) for x in v]) for v in per_kernel.values())
        busy = max(np.mean([x.get("lts__d_atomic_input_cycles_active.avg.pct_of_peak_sustained_elapsed", 0)
                            for x in v]) for v in per_kernel.values())
        src = NCU_SOURCES["forward" if name in ("clear", "depth", "accumulate", "normalize") else "backward"]
        h = hashlib.sha1()
        for rel in src:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        out[name] = {"kernel": " + ".join(sorted(per_kernel)), "launches_captured": sum(len(v) for v in per_kernel.values()),
                     "dram_bytes_per_launch": int(round(dram)), "l2_atomic_requests_per_launch": int(round(atom)),
                     "l2_atomic_unit_active_pct": round(float(busy), 2),
                     "ncu_duration_us": round(float(dur) / 1e3, 2),  # gpu__time_duration.sum is in ns
                     "sources": src, "sources_sha1": h.hexdigest()}
    return out


def atomic_peaks(device, px: int, ops: int = 1 << 26) -> dict:
    """Random-address atomic throughput on buffers the size of the 1080p
    pyramid's key, count and sum buffers (adop_atomic_probe, CUDA events,
    best of 3): the ceiling for the depth and accumulate passes, in atomics
    per second (one L2 request each, as the addresses are random)."""
    import torch
    import paper_2110_06635_gb300 as adop
    out = {}
    for name, kind, dt, elems, per in (("atomic_min_u64", 0, torch.int64, px, 1), ("atomic_add_u32", 1, torch.int32, px, 1),
                                       ("atomic_add_f32x4", 2, torch.float32, 2 * px, 4)):
        buf = torch.zeros(elems * per, dtype=dt, device=device)
        adop.adop_atomic_probe(kind, buf, elems, ops, 7)
        best = float("inf")
        for r in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            adop.adop_atomic_probe(kind, buf, elems, ops, 11 + r)
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        out[name] = round(ops / (best * 1e-3), 1)
        del buf
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------

def s8d_point_bytes(c: int, s_feat: int, recompute: bool = False):
    """Algorithmic bytes per point of one camera (the work unit: one point
    through all layers, forward + backward), as the measurement plan counts
    them: the forward reads xyz twice (depth and accumulate passes, 12 B
    each) and the descriptors once (c * s_feat); the backward reads xyz and
    the descriptors once and writes dL/dtau (4 c) and dL/dx (12), plus 12 B
    if the depth pass is re-run.  Returns (forward, backward)."""
    return 24 + c * s_feat, 24 + c * s_feat + 4 * c + (12 if recompute else 0)


def s8d_pixel_bytes(c: int, s_out: int):
    """Algorithmic bytes per pyramid pixel: the forward clears the key (8),
    count (4) and sums (4 c), then reads count and sums (4 + 4 c) and writes
    the image (c * s_out); the backward reads the upstream gradient (4 c).
    Returns (forward, backward)."""
    return (8 + 4 + 4 * c) + (4 + 4 * c) + c * s_out, 4 * c


def s8d_step_bytes(n: int, px: int, c: int, s_feat: int, s_out: int, recompute: bool = False) -> int:
    """Algorithmic bytes of one forward + backward of one camera."""
    pf, pb = s8d_point_bytes(c, s_feat, recompute)
    xf, xb = s8d_pixel_bytes(c, s_out)
    return n * (pf + pb) + px * (xf + xb)


def s8d_kernel_bytes(kernel: str, n: int, px: int, c: int, s_feat: int, s_out: int) -> int:
    """The same bytes split over the kernels that move them (per launch, one
    camera): the clear writes the per-pixel state, the depth pass reads xyz,
    the accumulate pass xyz and the descriptors, normalize the sums and the
    image, and the backward point pass every per-point read and write of the
    backward plus the upstream gradient (which it reads through the
    prepass's pixel-major copy).  Kernels that exist only in this design
    (prepass, binning, reduction) carry none: what they move is the
    implementation's own traffic (implementation_bytes)."""
    return {
        "clear": px * (8 + 4 + 4 * c),
        "depth": n * 12,
        "accumulate": n * (12 + c * s_feat),
        "normalize": px * (4 + 4 * c + c * s_out),
        "bwd_points": n * (24 + c * s_feat + 4 * c) + px * 4 * c,
    }.get(kernel, 0)


def bin_table_bytes(w: int, h: int, sms: int, ncam: int = 1) -> int:
    """Bytes of the binning's [block][tile] table for one camera: one 4-byte
    entry per block and 32x32-pixel tile, 8 blocks per SM shared by the
    cameras of a launch (at most 1536 rows in all)."""
    tiles = ((w + 31) // 32) * ((h + 31) // 32)
    rows = min((sms * 8 + ncam - 1) // ncam, (1536 + ncam - 1) // ncam)
    return rows * tiles * 4


def implementation_bytes(kernel: str, n: int, px: int, c: int, s_feat: int, s_out: int,
                         n_vis: int | None = None, bin_table: int = 0) -> int:
    """What one launch of this implementation must move (every buffer it
    touches read or written once), including its own records -- the keys it
    reads back, the backward's 16 B pixel records and pixel-major gradient,
    the layer masks and the binning lists.  Not algorithmic bytes: reported
    beside them to show where the design adds traffic (n points, px pyramid
    pixels, c channels, n_vis points in Lambda of at least one layer,
    bin_table bytes of the binning's block table)."""
    gs = c if c <= 2 else (c + 3) // 4 * 4
    nv = n if n_vis is None else n_vis
    return {
        "clear": px * (8 + 4 + 4 * c),                          # write key, count, sums
        "depth": n * (12 + 1) + px * 8 * 2,                     # read xyz -> layer byte; read+write keys
        "accumulate": n * (12 + 1 + c * s_feat + 4) + px * (8 + 2 * (4 + 4 * c)),  # xyz, byte, tau -> mask; keys; RMW count+sums
        "normalize": px * (4 + 4 * c + c * s_out),              # read count, sums; write image
        "bwd_prepass": px * (8 + 4 + 4 * c + 4 * c + 16 + 4 * gs),  # key, count, sums, G -> info, G'
        "bwd_bin": n * 8 + nv * 4 + 2 * bin_table,                    # masks twice -> list; table written, read
        # list, mask, xyz, tau -> grads of the visible points; pixel records; masks -> zero grads of the rest
        "bwd_points": nv * (4 + 4 + 12 + c * s_feat + 4 * c + 12) + px * (16 + 4 * gs) + n * 4 + (n - nv) * (4 * c + 12),
        "bwd_reduce": 0,
    }.get(kernel, 0)


def kernel_roofline(ks: dict, n: int, px: int, c: int, s_feat: int, s_out: int, n_vis: int, peak: float,
                    peak_kind: str, kernel: str | None = None, recorded: bool = True) -> dict:
    """Roofline of one kernel (default: the one with the most device time):
    its algorithmic bytes per launch over its average CUDA-event launch time,
    against the measured HBM copy bandwidth; beside it the same for the bytes
    this implementation moves (implementation_bytes).  `traffic` is the ncu
    DRAM record of the headline workload, so other workloads pass
    recorded=False."""
    dom = kernel or max(ks, key=lambda k: ks[k][1])
    launches, dom_ms = ks[dom]
    ab = s8d_kernel_bytes(dom, n, px, c, s_feat, s_out)
    ib = implementation_bytes(dom, n, px, c, s_feat, s_out, n_vis)
    t = dom_ms / launches * 1e-3
    achieved = ab / t / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "traffic": recorded_traffic(dom) if recorded else None,
            "algorithmic_bytes_per_launch": ab,
            "implementation_bytes_per_launch": ib,
            "frac_implementation_bytes": round(ib / t / 1e9 / peak, 4),
            "avg_launch_ms": round(dom_ms / launches, 4)}


class Workload:
    def __init__(self, n_points: int, feat_dtype: str, device: str, scene=None, cam=None, discard: bool = False,
                 env: bool = False, grad_io: str = "f32"):
        import torch
        import paper_2110_06635_gb300 as adop
        import scenes
        self.adop = adop
        if scene is None:
            scene, cams = scenes.config(2, n=n_points)
            cam = cams[0]
        self.scene, self.cam = scene, cam
        self.n, self.c = scene.n, scene.c
        self.device = device
        self.feat_dtype = feat_dtype
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[feat_dtype]
        self.xyz = torch.from_numpy(scene.xyz).to(device)
        if feat_dtype == "bf16":
            self.feat = torch.from_numpy(scene.feat_as("bf16").view(np.int16)).to(device).view(torch.bfloat16)
        else:
            self.feat = torch.from_numpy(scene.feat).to(device)
        self.out_dtype = tdt
        self.radius = self.beta = None
        flags = adop.ADOP_FLAG_GRAD_ASSIGN
        if discard:
            # the paper's preprocess (4th-nearest-point radius) and a fixed uniform draw per point
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.radius = adop.adop_point_radius(self.xyz, 4)
            torch.cuda.synchronize()
            self.radius_ms = (time.perf_counter() - t0) * 1e3
            g = torch.Generator(device=device).manual_seed(1234)
            self.beta = torch.rand(scene.n, generator=g, device=device)
            flags |= adop.ADOP_FLAG_DISCARD
        self.pts = adop.Points(self.xyz, self.feat, None, self.radius, self.beta)
        self.env = self.genv = None
        if env:
            # the paper's 1024^2 spherical map of neural features, read as equirectangular
            E = scenes.env_map(self.c, 1024, 1024, seed=2025)
            self.env = torch.from_numpy(np.ascontiguousarray(np.moveaxis(E, 0, -1))).to(device)
            self.genv = torch.zeros_like(self.env)
        self.params = adop.Params(LEVELS, 0.01, 1e-3, None, flags, 1.5, self.env)
        self.frame = adop.Frame.alloc(cam, self.c, LEVELS, tdt, True, device, self.n)
        self.ws = adop.alloc_workspace(self.pts, [cam], self.params, None, device)
        G = scenes.upstream_grad(cam.w, cam.h, LEVELS, self.c, 2024)
        self.G_host = G
        # gradient storage: FP32, or ("bf16") the upstream gradients and dL/dtau
        # in BF16 (summed in FP32 on the device, rounded once)
        self.grad_dt = {"f32": torch.float32, "bf16": torch.bfloat16}[grad_io]
        self.G = [torch.from_numpy(g).to(device).to(self.grad_dt) for g in G]
        self.gfeat = torch.empty((self.n, self.c), dtype=self.grad_dt, device=device)
        self.gxyz = torch.empty((self.n, 3), dtype=torch.float32, device=device)
        self.gpose = torch.zeros((1, 6), dtype=torch.float32, device=device)
        self.gintr = torch.zeros((1, 6), dtype=torch.float32, device=device)
        self.px = adop.pyramid_offsets(cam.w, cam.h, LEVELS)[-1]
        self.bin_table = bin_table_bytes(cam.w, cam.h, torch.cuda.get_device_properties(device).multi_processor_count)
        self.s_feat = 2 if feat_dtype == "bf16" else 4
        self._prepare()

    def _prepare(self):
        """Marshal the C structs once, so a step is two foreign calls."""
        import ctypes as ct
        from paper_2110_06635_gb300 import _abi as A
        lib = A.load()
        self._lib = lib
        self._ps = self.pts.struct()
        self._pr = self.params.struct()
        self._pr.grad_dtype = A.dtype_code(self.grad_dt)
        self._pr.grad_feat_dtype = A.dtype_code(self.grad_dt)
        self._cams = A._cams_array([self.cam])
        self._fr = (A.adop_frame * 1)(self.frame.struct())
        self._g = (ct.c_void_p * LEVELS)(*[g.data_ptr() for g in self.G])
        self._wp, self._wn = A._ws_ptr(self.ws)
        self._ct = ct

    def graph_step(self):
        """One step captured in a CUDA graph; returns the replay callable."""
        import torch
        ct = self._ct
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(ct.c_void_p(side.cuda_stream))
        torch.cuda.current_stream().wait_stream(side)
        self._graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self._graph):
            self.step(ct.c_void_p(torch.cuda.current_stream().cuda_stream))
        return self._graph.replay

    def step(self, stream_ptr):
        ct = self._ct
        st = self._lib.adop_render_forward(ct.byref(self._ps), self._cams, 1, ct.byref(self._pr), self._fr,
                                           self._wp, self._wn, stream_ptr)
        if st != 0:
            raise RuntimeError(self._lib.adop_last_error().decode())
        st = self._lib.adop_render_backward(ct.byref(self._ps), self._cams, 1, ct.byref(self._pr), self._fr,
                                            self._g, self.gfeat.data_ptr(), self.gxyz.data_ptr(),
                                            self.gpose.data_ptr(), self.gintr.data_ptr(), self._wp, self._wn,
                                            stream_ptr)
        if st != 0:
            raise RuntimeError(self._lib.adop_last_error().decode())
        if self.env is not None:
            st = self._lib.adop_env_backward(self._cams, 1, ct.byref(self._pr), self.c, self._fr, self._g,
                                             self.genv.data_ptr(), stream_ptr)
            if st != 0:
                raise RuntimeError(self._lib.adop_last_error().decode())


def run_ours(args, dist, rank, world):
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    adop.build()
    adop.load()
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def flush():
        flush_buf.zero_()

    stream = torch.cuda.current_stream()
    sp = ct.c_void_p(stream.cuda_stream)
    results = {}
    dtypes = ["bf16"] if (args.no_fp32 or args.profile_only) else ["bf16", "f32"]
    clocks = None
    for dt in dtypes:
        wl = Workload(args.points, dt, device)
        for _ in range(args.warmup):
            wl.step(sp)
        torch.cuda.synchronize()
        wl.n_vis = int(((wl.frame.vis & 0xFF) != 0).sum().item())
        # per-kernel times: the eager step with the library's launch events
        adop.adop_profile_enable(True)
        adop.adop_profile_collect()
        eager_ms, _ = timed_steps(lambda: wl.step(sp), args.steps, flush, dist, device)
        kstats = adop.adop_profile_collect()
        adop.adop_profile_enable(False)
        # the timed steps: the same step captured once in a CUDA graph and
        # replayed (the same launches on the same buffers, without the host's
        # launch gaps between the kernels)
        step = (lambda: wl.step(sp)) if args.eager else wl.graph_step()
        for _ in range(2):
            step()
        sampler = ClockSampler(gpu_index(device))
        with sampler:
            total_ms, per = timed_steps(step, args.steps, flush, dist, device)
        if dt == "bf16":
            clocks = sampler.summary()
        tmax = max_over_ranks(dist, total_ms, device)
        results[dt] = {"wl": wl, "total_ms": tmax, "per": per, "kstats": kstats,
                       "eager_ms": max_over_ranks(dist, eager_ms, device)}
        if dt != dtypes[-1]:
            del wl
            torch.cuda.empty_cache()
    return results, clocks, device


def bench_shuffled(device, steps: int, warmup: int, flush) -> dict:
    """The headline workload with its points in a random order instead of
    surface by surface (the paper sorts its clouds for locality): how much the
    point order is worth.  The step is the same eager step as `kernel_ms`."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    import scenes
    sc, cams = scenes.config(2, shuffle=True)
    wl = Workload(sc.n, "bf16", device, scene=sc, cam=cams[0])
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(warmup):
        wl.step(sp)
    adop.adop_profile_enable(True)
    adop.adop_profile_collect()
    total_ms, _ = timed_steps(lambda: wl.step(sp), steps, flush, None, device)
    ks = adop.adop_profile_collect()
    adop.adop_profile_enable(False)
    out = {"workload": "the headline view with the 5M points in a random order",
           "value": round(wl.n * steps / (total_ms / 1e3), 1), "unit": UNIT,
           "ms_per_step": round(total_ms / steps, 4),
           "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()}}
    del wl
    torch.cuda.empty_cache()
    return out


def bench_discard(device, steps: int, warmup: int, flush) -> dict:
    """The headline workload with stochastic point discarding (Eq. discard,
    gamma = 1.5, the paper's timed configuration): r_world from the 4th
    nearest point (GPU preprocess, timed separately), beta ~ U[0,1) fixed."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    wl = Workload(5_000_000, "bf16", device, discard=True)
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(warmup):
        wl.step(sp)
    torch.cuda.synchronize()
    m = wl.frame.vis & 0xFF
    kept = [float(((m >> l) & 1).sum().item()) for l in range(LEVELS)]
    adop.adop_profile_enable(True)
    adop.adop_profile_collect()
    total_ms, _ = timed_steps(lambda: wl.step(sp), steps, flush, None, device)
    ks = adop.adop_profile_collect()
    adop.adop_profile_enable(False)
    out = {"workload": "the headline view with stochastic discarding, gamma = 1.5",
           "value": round(wl.n * steps / (total_ms / 1e3), 1), "unit": UNIT,
           "ms_per_step": round(total_ms / steps, 4),
           "points_in_lambda_per_layer": kept,
           "radius_preprocess_ms": round(wl.radius_ms, 2),
           "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()}}
    del wl
    torch.cuda.empty_cache()
    return out


def bench_env(device, steps: int, warmup: int, flush) -> dict:
    """The headline workload with an environment map (Sec. 3.1): a 1024 x 1024
    equirectangular map of C = 8 FP32 features sampled for the empty pixels,
    and its gradient (adop_env_backward) in every step."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    wl = Workload(5_000_000, "bf16", device, env=True)
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(warmup):
        wl.step(sp)
    torch.cuda.synchronize()
    empty = float((wl.frame.count == 0).float().mean().item())
    adop.adop_profile_enable(True)
    adop.adop_profile_collect()
    total_ms, _ = timed_steps(lambda: wl.step(sp), steps, flush, None, device)
    ks = adop.adop_profile_collect()
    adop.adop_profile_enable(False)
    out = {"workload": "the headline view with a 1024x1024 C=8 environment map and its gradient",
           "value": round(wl.n * steps / (total_ms / 1e3), 1), "unit": UNIT,
           "ms_per_step": round(total_ms / steps, 4), "empty_pixel_fraction": round(empty, 4),
           "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()}}
    del wl
    torch.cuda.empty_cache()
    return out


def e2e_measure(wl, steps: int, warmup: int, device):
    """The same step through the public API from and to pinned host memory
    (paper_2110_06635_gb300.pipeline): every step copies its positions,
    descriptors and upstream gradients host -> device and its images and all
    gradients device -> host; the copies of neighbouring steps overlap the
    kernels on separate streams.  Timed with CUDA events from before the first
    copy to after the last."""
    import torch
    from paper_2110_06635_gb300.pipeline import HostPipeline, StepIO
    pipe = HostPipeline(wl.cam, wl.n, wl.c, wl.feat.dtype, wl.out_dtype, LEVELS, device=device,
                        grad_dtype=wl.grad_dt, grad_feat_dtype=wl.grad_dt)
    ios = [StepIO.alloc(wl.cam, wl.n, wl.c, wl.feat.dtype, wl.out_dtype, LEVELS, grad_dtype=wl.grad_dt,
                        grad_feat_dtype=wl.grad_dt) for _ in range(2)]
    for io in ios:  # two host input sets, used alternately (each step still moves its own bytes)
        io.xyz.copy_(wl.xyz.cpu())
        io.feat.copy_(wl.feat.cpu())
        for h, d in zip(io.grads, wl.G):
            h.copy_(d.cpu())
    pipe.run([ios[k % 2] for k in range(warmup)])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pipe.run([ios[k % 2] for k in range(steps)], start=a, end=b)
    b.synchronize()
    total_ms = a.elapsed_time(b)
    del pipe
    return total_ms, ios[0].bytes_in(), ios[0].bytes_out()


def _oracle_step(oracle, sc, feat, cam, Gf, idx, threads):
    """One oracle forward + backward of the workload's points idx (None = all)."""
    xyz, fe = (sc.xyz, feat) if idx is None else (sc.xyz[idx], feat[idx])
    f = oracle.forward(xyz, fe, cam, LEVELS, 0.01, 1e-3, threads=threads)
    oracle.backward(f, xyz, fe, cam, Gf, 0.01, threads=threads)


def bench_bf16_io(device, steps: int, warmup: int, flush) -> dict:
    """The headline step with BF16 upstream gradients and BF16 dL/dtau (what
    a BF16 training step hands the rasterizer and expects back: the library
    widens the gradients to FP32, sums dL/dtau in FP32 and rounds it once),
    timed on the device as a CUDA graph and end to end from host buffers."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    wl = Workload(5_000_000, "bf16", device, grad_io="bf16")
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(warmup):
        wl.step(sp)
    adop.adop_profile_enable(True)
    adop.adop_profile_collect()
    timed_steps(lambda: wl.step(sp), steps, flush, None, device)
    ks = adop.adop_profile_collect()
    adop.adop_profile_enable(False)
    step = wl.graph_step()
    for _ in range(2):
        step()
    total_ms, _ = timed_steps(step, steps, flush, None, device)
    ksteps = max(30, steps)
    e2e_ms, bi, bo = e2e_measure(wl, ksteps, 2, device)
    out = {"workload": "the headline step with the upstream gradients and dL/dtau stored in BF16",
           "value": round(wl.n * steps / (total_ms / 1e3), 1), "unit": UNIT,
           "ms_per_step": round(total_ms / steps, 4),
           "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()},
           "e2e": {"value": round(wl.n * ksteps / (e2e_ms / 1e3), 1), "unit": UNIT, "h2d_bytes_per_step": bi,
                   "d2h_bytes_per_step": bo, "steps": ksteps}}
    del wl
    torch.cuda.empty_cache()
    return out


def cpu_baseline(budget_s: float = 10.0):
    """The oracle as it stands on the host, on the same camera and 1080p
    pyramid: on every core (its forward splits the pixels, its backward the
    points, over OpenMP threads) over the whole 5M-point workload, repeated
    for about budget_s; and on one thread over random 500K-point samples of
    it, for about budget_s."""
    import oracle
    import scenes
    sc, cams = scenes.config(2)
    cam = cams[0]
    feat = sc.feat_as("bf16")
    G = scenes.upstream_grad(cam.w, cam.h, LEVELS, sc.c, 2024)
    Gf = np.concatenate([g.ravel() for g in G]).astype(np.float64)
    cores = oracle.threads(0)
    done, t_used, reps = 0, 0.0, 0
    while t_used < budget_s and reps < 64:
        t0 = time.perf_counter()
        _oracle_step(oracle, sc, feat, cam, Gf, None, 0)
        t_used += time.perf_counter() - t0
        done += sc.n
        reps += 1
    allcore = {"value": round(done / t_used, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the whole 5M-point workload, {reps} forward+backward passes, full 1920x1080 4-layer "
                         f"pyramid, FP64 C oracle on {cores} OpenMP threads, {t_used:.1f} s"}
    rng = np.random.default_rng(99)
    m = 500_000
    done, t_used, reps = 0, 0.0, 0
    while t_used < budget_s and reps < 64:
        idx = np.sort(rng.choice(sc.n, size=min(m, sc.n), replace=False))
        t0 = time.perf_counter()
        _oracle_step(oracle, sc, feat, cam, Gf, idx, 1)
        t_used += time.perf_counter() - t0
        done += len(idx)
        reps += 1
    allcore["single_thread"] = {
        "value": round(done / t_used, 1), "unit": UNIT, "cores": 1,
        "sample": f"{reps} x {m} points drawn from the 5M-point workload, full 1920x1080 4-layer pyramid, "
                  f"fwd+bwd, FP64 C oracle, one thread, {t_used:.1f} s"}
    return allcore


# ---------------------------------------------------------------------------
# further workloads, reported beside the headline number
# ---------------------------------------------------------------------------

def bench_training_step(device, steps: int = 5, warmup: int = 3) -> dict:
    """20M points, C=8 BF16, 16 orbit cameras 960x540..1920x1080 with their own
    exposure / white balance / vignette / response curve, forward + backward of
    all 16 through the autograd.Function, depth pass re-rendered in backward
    (no per-pixel state kept), FP32 gradient accumulation across cameras."""
    import torch
    import paper_2110_06635_gb300 as adop
    import scenes
    from paper_2110_06635_gb300.autograd import rasterize
    sc, cams = scenes.config(3)
    xyz = torch.from_numpy(sc.xyz).to(device).requires_grad_()
    feat = torch.from_numpy(sc.feat_as("bf16").view(np.int16)).to(device).view(torch.bfloat16).requires_grad_()
    luts = [torch.from_numpy(np.ascontiguousarray(c.crf, np.float32)).to(device) for c in cams]
    xi = torch.zeros((len(cams), 6), dtype=torch.float32, device=device, requires_grad=True)
    G = [[torch.randn(sc.c, c.h >> l, c.w >> l, device=device, generator=torch.Generator(device).manual_seed(k))
          .to(torch.bfloat16) for l in range(LEVELS)] for k, c in enumerate(cams)]
    flat_g = [g for row in G for g in row]

    def step():
        imgs = rasterize(xyz, feat, cams, xi, levels=LEVELS, flags=adop.ADOP_FLAG_EPILOGUE,
                         out_dtype=torch.bfloat16, keep_state=False, crf_luts=luts)
        torch.autograd.backward([im for row in imgs for im in row], flat_g)

    for _ in range(warmup):
        step()
    adop.adop_profile_enable(True)
    adop.adop_profile_collect()
    total_ms, per = timed_steps(step, steps, None, None, device)
    ks = adop.adop_profile_collect()
    adop.adop_profile_enable(False)
    views = len(cams)

    # the alternative design: one camera per call (owner-computes gradients,
    # no atomics across cameras), the cameras one after another
    def step_by_camera():
        for k in range(views):
            imgs = rasterize(xyz, feat, cams[k:k + 1], xi[k:k + 1], levels=LEVELS, flags=adop.ADOP_FLAG_EPILOGUE,
                             out_dtype=torch.bfloat16, keep_state=False, crf_luts=luts[k:k + 1])
            torch.autograd.backward(imgs[0], G[k])

    for _ in range(2):
        step_by_camera()
    seq_ms, _ = timed_steps(step_by_camera, steps, None, None, device)
    px = sum(adop.pyramid_offsets(c.w, c.h, LEVELS)[-1] for c in cams)
    peak, peak_kind = measured_peaks()
    ms = total_ms / steps
    # algorithmic bytes of the step: every view's forward + backward with the
    # depth pass re-run (the plan's +12 B per point), and every view's pixels
    sb = sum(s8d_step_bytes(sc.n, adop.pyramid_offsets(c.w, c.h, LEVELS)[-1], sc.c, 2, 2, recompute=True)
             for c in cams)
    per_launch = {k: (v[1] / v[0]) for k, v in ks.items()}
    roof = {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
            "step_bytes_algorithmic": sb, "step_achieved": round(sb / (ms * 1e-3) / 1e9, 1),
            "step_frac": round(sb / (ms * 1e-3) / 1e9 / peak, 4)}
    for k, b in (("depth", views * sc.n * 12), ("accumulate", views * sc.n * (12 + sc.c * 2))):
        if k in per_launch:  # each launch renders all views: b bytes of points per launch
            roof[k] = {"ms_per_launch": round(per_launch[k], 4), "ms_per_view": round(per_launch[k] / views, 4),
                       "achieved": round(b / (per_launch[k] * 1e-3) / 1e9, 1),
                       "frac": round(b / (per_launch[k] * 1e-3) / 1e9 / peak, 4)}
    out = {"workload": f"{sc.n} points C=8 BF16, {views} cameras 960x540..1920x1080 ({px} pyramid px), "
                       "fwd+bwd via autograd, epilogue on, depth re-rendered in backward",
           "roofline": roof,
           "ms_per_step": round(total_ms / steps, 3),
           "ms_per_step_camera_by_camera": round(seq_ms / steps, 3),
           "point_views_per_s": round(sc.n * views * steps / (total_ms / 1e3), 1),
           "gpu_launches_per_step": round(sum(v[0] for v in ks.values()) / steps, 2),
           "kernel_ms_per_step": {k: round(v[1] / steps, 3) for k, v in ks.items()}}
    del xyz, feat, G, flat_g
    torch.cuda.empty_cache()
    return out


def bench_large_fwd_bwd(device, sc, steps: int, warmup: int, flush, dtypes=("bf16", "f32")) -> dict:
    """Forward + backward of one 1920x1080 view of the 120M-point cloud (the
    large scene's first path camera), C = 4 descriptors stored in BF16 and in
    FP32, gradients to descriptors, positions, pose and intrinsics: the same
    step as the headline (kept state, gradients assigned), captured once as a
    CUDA graph and replayed, L2 flushed between steps.  The roofline is the
    step's algorithmic bytes over its time, and the dominant kernel's."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    import scenes
    cam = scenes.path_cameras(60, 1920, 1080, seed=1004)[0]
    peak, peak_kind = measured_peaks()
    sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {"workload": f"{sc.n} points on 500 surfaces in a 100 m box, C=4, one 1920x1080 view of the "
                       "60-frame path, 4 layers, fwd+bwd to tau, x, pose, intrinsics",
           "points": sc.n, "resolution": "1920x1080"}
    for dt in dtypes:
        wl = Workload(sc.n, dt, device, scene=sc, cam=cam)
        for _ in range(warmup):
            wl.step(sp)
        torch.cuda.synchronize()
        n_vis = int(((wl.frame.vis & 0xFF) != 0).sum().item())
        adop.adop_profile_enable(True)
        adop.adop_profile_collect()
        eager_ms, _ = timed_steps(lambda: wl.step(sp), steps, flush, None, device)
        ks = adop.adop_profile_collect()
        adop.adop_profile_enable(False)
        step = wl.graph_step()
        for _ in range(2):
            step()
        total_ms, _ = timed_steps(step, steps, flush, None, device)
        ms = total_ms / steps
        sb = s8d_step_bytes(wl.n, wl.px, wl.c, wl.s_feat, wl.s_feat)
        out[dt] = {"ms_per_step": round(ms, 4), "ms_per_step_eager": round(eager_ms / steps, 4),
                   "value": round(wl.n / (ms * 1e-3), 1), "unit": UNIT,
                   "points_in_lambda": n_vis, "step_bytes_algorithmic": sb,
                   "step_hbm_fraction": round(sb / (ms * 1e-3) / 1e9 / peak, 4),
                   "roofline": kernel_roofline(ks, wl.n, wl.px, wl.c, wl.s_feat, wl.s_feat, n_vis, peak, peak_kind,
                                               recorded=False),
                   "step_bytes_implementation": sum(implementation_bytes(k, wl.n, wl.px, wl.c, wl.s_feat, wl.s_feat,
                                                                         n_vis, wl.bin_table) * ks[k][0]
                                                    for k in ks) // steps,
                   "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()}}
        del wl, step
        torch.cuda.empty_cache()
    return out


def bench_large_scene(device, sc, frames: int = 60) -> dict:
    """120M points (FP32 xyz + 4-channel FP16 descriptors, 2.4 GB) on 500
    surfaces in a 100 m box; forward only along a 60-frame path at 1920x1080
    and 3840x2160; 4 layers, alpha = 0.01."""
    import ctypes as ct
    import torch
    import paper_2110_06635_gb300 as adop
    import scenes
    from paper_2110_06635_gb300 import _abi as A
    xyz = torch.from_numpy(sc.xyz).to(device)
    feat = torch.from_numpy(sc.feat.astype(np.float16)).to(device)
    n = sc.n
    pts = adop.Points(xyz, feat)
    params = adop.Params(LEVELS, 0.01, 1e-3, None, 0)
    res = {}
    peak, _ = measured_peaks()
    for (w, h) in ((1920, 1080), (3840, 2160)):
        cams = scenes.path_cameras(frames, w, h, seed=1004)
        fr = adop.Frame.alloc(cams[0], 4, LEVELS, torch.float16, False, device)
        ws = adop.alloc_workspace(pts, [cams[0]], params, None, device)
        lib = A.load()
        ps, pr = pts.struct(), params.struct()
        frs = (A.adop_frame * 1)(fr.struct())
        wp, wn = A._ws_ptr(ws)
        sp = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        carr = [A._cams_array([c]) for c in cams]
        it = iter(range(10 ** 9))

        def step():
            k = next(it) % frames
            st = lib.adop_render_forward(ct.byref(ps), carr[k], 1, ct.byref(pr), frs, wp, wn, sp)
            if st != 0:
                raise RuntimeError(lib.adop_last_error().decode())

        for _ in range(3):
            step()
        adop.adop_profile_enable(True)
        adop.adop_profile_collect()
        total_ms, _ = timed_steps(step, frames, None, None, device)
        ks = adop.adop_profile_collect()
        adop.adop_profile_enable(False)
        px = adop.pyramid_offsets(w, h, LEVELS)[-1]
        fb = n * s8d_point_bytes(4, 2)[0] + px * s8d_pixel_bytes(4, 2)[0]  # forward bytes (FP16 in, FP16 out)
        ms = total_ms / frames
        res[f"{w}x{h}"] = {"fps": round(1e3 / ms, 2), "ms_per_frame": round(ms, 3),
                           "points_per_s": round(n / (ms / 1e3), 1),
                           "hbm_fraction_of_measured": round(fb / (ms * 1e-3) / 1e9 / peak, 4),
                           "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in ks.items()}}
        del ws, fr
        torch.cuda.empty_cache()
    del xyz, feat, pts
    torch.cuda.empty_cache()
    return {"workload": f"{n} points FP32 xyz + C=4 FP16, 60-frame path, forward only, 4 layers", **res}


def bench_serving(device, seconds: float = 4.0, rates=(200.0, 1000.0, 2000.0), outstanding: int = 64) -> dict:
    """Three resident clouds (1M, 10M, 50M points, C=8); requests of random
    orbit views at 640x480 / 1280x720 / 1920x1080 / 3840x2160 (uniform) over
    a uniformly drawn cloud, forward + photometric epilogue.  Two servers:
    (i) continuous batching, BF16 descriptors and output (64 slots, 4
    streams, up to 8 cameras of any clouds per launch); (ii) one request at a
    time, FP32.  Each is measured under Poisson arrivals at each rate and in
    a closed loop that keeps `outstanding` requests in flight (the saturated
    throughput), for `seconds` after a 1 s warm-up.  Latency = submit to
    device completion.  Output buffers come from a ring of 16 per
    resolution; a request whose buffer is still in use waits for it (the
    time the client spent blocked is reported: at rates beyond a server's
    capacity the queue would otherwise grow without bound)."""
    import torch
    import paper_2110_06635_gb300 as adop
    import scenes
    res_set = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))
    ring = 16
    base = [scenes.surfaces_scene(n, 8, seed=1005 + k, size_scale=scenes.SIZE_SCALE_SINGLE_VIEW)
            for k, n in enumerate((1_000_000, 10_000_000, 50_000_000))]
    lut = torch.from_numpy(scenes.crf_gamma_lut()).to(device)
    rng0 = np.random.default_rng(2026)
    pool = []  # a fixed pool of requests, cycled
    for _ in range(512):
        w, h = res_set[int(rng0.integers(4))]
        cam = scenes.orbit_cameras(1, seed=int(rng0.integers(1 << 30)), resolutions=((w, h),))[0]
        pool.append((int(rng0.integers(3)), res_set.index((w, h)), cam))
    out = {}
    for mode in ("bf16_batched", "fp32_unbatched"):
        bf16 = mode.startswith("bf16")
        dt = torch.bfloat16 if bf16 else torch.float32
        clouds = []
        for sc in base:
            f = torch.from_numpy(sc.feat_as("bf16").view(np.int16)).to(device).view(torch.bfloat16) if bf16 \
                else torch.from_numpy(sc.feat).to(device)
            clouds.append(adop.Points(torch.from_numpy(sc.xyz).to(device), f))
        bufs = [[torch.empty(adop.output_numel(scenes.Camera(w, h, 1.0, 1.0, 0.0, 0.0), 8, LEVELS), dtype=dt,
                             device=device) for _ in range(ring)] for (w, h) in res_set]
        srv = adop.Server(mem_budget_bytes=8 << 30, max_slots=64 if bf16 else 1, streams=4 if bf16 else 1,
                          max_batch=8 if bf16 else 1, levels=LEVELS, flags=adop.ADOP_FLAG_EPILOGUE, out_dtype=dt)
        ids = [srv.load_cloud(p) for p in clouds]
        owner = [[None] * ring for _ in res_set]  # ticket last rendered into each buffer
        nxt = [0] * len(res_set)
        state = {"k": 0, "blocked": 0.0}

        def submit():
            cid, ri, cam = pool[state["k"] % len(pool)]
            state["k"] += 1
            j = nxt[ri] % ring
            nxt[ri] += 1
            if owner[ri][j] is not None:
                t0 = time.perf_counter()
                srv.wait(owner[ri][j], 120_000)
                state["blocked"] += time.perf_counter() - t0
            t = srv.submit(ids[cid], cam, bufs[ri][j], lut)
            owner[ri][j] = t
            return t

        def drain():
            for row in owner:
                for t in row:
                    if t is not None:
                        srv.wait(t, 120_000)

        res = {}
        for rate in list(rates) + ["saturated"]:
            rng = np.random.default_rng(7)
            for phase in ("warm", "measure"):
                dur = 1.0 if phase == "warm" else seconds
                state["blocked"] = 0.0
                t0 = time.perf_counter()
                if rate == "saturated":
                    inflight = []
                    while time.perf_counter() - t0 < dur:
                        while len(inflight) >= outstanding:
                            srv.wait(inflight.pop(0), 120_000)
                        inflight.append(submit())
                else:
                    ta = t0
                    while ta - t0 < dur:
                        ta += rng.exponential(1.0 / rate)
                        d = ta - time.perf_counter()
                        if d > 0:
                            time.sleep(d)
                        submit()
                drain()
                if phase == "warm":
                    srv.reset_stats()
            st = srv.stats()
            key = "saturated" if rate == "saturated" else f"poisson_{int(rate)}"
            res[key] = {"offered_req_per_s": None if rate == "saturated" else rate,
                        "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                        "mean_ms": round(st["mean_ms"], 3), "max_ms": round(st["max_ms"], 3),
                        "req_per_s": round(st["req_per_s"], 1), "points_per_s": round(st["points_per_s"], 1),
                        "completed": st["completed"], "mean_batch": round(st["mean_batch"], 2),
                        "mixed_cloud_batches": st["mixed_batches"],
                        "client_blocked_s": round(state["blocked"], 3)}
            if rate == "saturated":
                res[key]["outstanding"] = outstanding
        res["mem_peak_bytes"] = srv.stats()["mem_peak"]
        out[mode] = res
        srv.close()
        del clouds, bufs
        torch.cuda.empty_cache()
    out["workload"] = (f"clouds of 1M/10M/50M points (C=8), views at 640x480/1280x720/1920x1080/3840x2160 "
                       f"(uniform), forward + photometric epilogue; Poisson arrivals at {', '.join(str(int(r)) for r in rates)} "
                       f"req/s and a closed loop of {outstanding} outstanding requests, {seconds:.0f} s each after "
                       "1 s of warm-up")
    return out


def atomic_roofline(device, wl, ks) -> dict:
    """The second ceiling of the depth and accumulate passes: L2 atomics.
    Achieved = L2 atomic requests per launch (ncu, committed summary) / the
    launch's CUDA-event time; peak = the random-address probe's rate."""
    peaks = atomic_peaks(device, wl.px)
    out = {"unit": "L2 atomic requests/s", "peaks": peaks,
           "l2_bytes": int(getattr(__import__("torch").cuda.get_device_properties(device), "L2_cache_size", 0)),
           "pixel_state_bytes": wl.px * (8 + 4 + 4 * wl.c)}
    for name, peak_key in (("depth", "atomic_min_u64"), ("accumulate", "atomic_add_f32x4")):
        rec = recorded_atomics(name)
        if rec is None or name not in ks:
            out[name] = None
            continue
        req, busy = rec
        t = ks[name][1] / ks[name][0] * 1e-3
        out[name] = {"l2_atomic_requests_per_launch": req, "achieved": round(req / t, 1),
                     "peak": peaks[peak_key], "frac": round(req / t / peaks[peak_key], 4),
                     "l2_atomic_unit_active_pct_ncu": busy}
    return out


def main():
    args = parse()
    if args.record_traffic:
        rec = record_traffic(args.record_traffic)
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json"), "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(json.dumps({k: (v["dram_bytes_per_launch"], v["l2_atomic_requests_per_launch"]) for k, v in rec.items()}))
        return
    if args.impl == "reference":
        return main_reference(args)
    if args.profile_large:
        import torch
        import scenes
        torch.cuda.set_device(0)
        flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda:0")
        sc_large, _ = scenes.config(4)
        res = bench_large_fwd_bwd("cuda:0", sc_large, args.steps, args.warmup, flush_buf.zero_, dtypes=("bf16",))
        print(json.dumps({"large_scene_fwd_bwd": res}))
        return
    dist, rank, world = dist_setup()
    results, clocks, device = run_ours(args, dist, rank, world)
    bf = results["bf16"]
    wl = bf["wl"]
    K = args.steps
    ms_per_step = bf["total_ms"] / K
    value = world * wl.n * K / (bf["total_ms"] / 1e3)
    peak, peak_kind = measured_peaks()
    # dominant kernel by device time
    ks = bf["kstats"]
    roofline = kernel_roofline(ks, wl.n, wl.px, wl.c, wl.s_feat, 2, wl.n_vis, peak, peak_kind)
    kernel_ms = {k: round(v[1] / v[0], 4) for k, v in ks.items()}
    step_bytes = s8d_step_bytes(wl.n, wl.px, wl.c, wl.s_feat, 2)
    impl_step_bytes = sum(implementation_bytes(k, wl.n, wl.px, wl.c, wl.s_feat, 2, wl.n_vis, wl.bin_table) *
                          ks[k][0] for k in ks) // K
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "ms_per_step_eager": round(bf["eager_ms"] / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 storage, f32 arithmetic", "data": "synthetic",
        "config": {"workload": "single view 1920x1080: 5M points on 50 seeded surfaces (depth complexity ~8), "
                               "C=8 BF16 descriptors, 4 layers, alpha=0.01, fwd+bwd to tau, x, pose, intrinsics",
                   "points": wl.n, "resolution": "1920x1080", "channels": wl.c, "levels": LEVELS,
                   "feat_dtype": "bf16", "l2": "flushed between timed steps (256 MiB write, outside the events)",
                   "launch": "eager" if args.eager else "one step captured as a CUDA graph, replayed per step",
                   "points_in_lambda": wl.n_vis,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "atomic_roofline": None if args.profile_only else atomic_roofline(device, wl, ks),
        "kernel_ms": kernel_ms,
        "step_hbm_fraction": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4),
        "step_bytes": {"algorithmic": step_bytes, "implementation": impl_step_bytes,
                       "per_point": sum(s8d_point_bytes(wl.c, wl.s_feat)),
                       "per_pixel": sum(s8d_pixel_bytes(wl.c, 2))},
        "gpu_launches": int(sum(v[0] for v in ks.values())),
        "clocks": clocks,
    }
    if "f32" in results:
        f32 = results["f32"]
        line["fp32"] = {"value": round(world * f32["wl"].n * K / (f32["total_ms"] / 1e3), 1),
                        "ms_per_step": round(f32["total_ms"] / K, 4),
                        "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in f32["kstats"].items()}}
    if not args.no_e2e and not args.profile_only:
        # at least 30 steps: the pipeline's first input copy and last result
        # copy overlap nothing, and are spread over the steps like any other
        ksteps = max(30, K)
        e2e_ms, bi, bo = e2e_measure(wl, ksteps, 2, device)
        e2e_ms = max_over_ranks(dist, e2e_ms, device)
        line["e2e"] = {"value": round(world * wl.n * ksteps / (e2e_ms / 1e3), 1), "unit": UNIT,
                       "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "steps": ksteps}
    if not args.profile_only:
        bf = results = wl = None  # free the headline workload before the larger ones
        import torch
        torch.cuda.empty_cache()
        if not args.no_e2e:
            fb = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
            line["bf16_io"] = bench_bf16_io(device, args.steps, args.warmup, lambda: fb.zero_())
            del fb
        if not args.no_discard:
            fb = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
            line["stochastic_discard"] = bench_discard(device, args.steps, args.warmup, lambda: fb.zero_())
            del fb
        if not args.no_shuffle:
            fb = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
            line["shuffled_points"] = bench_shuffled(device, args.steps, args.warmup, lambda: fb.zero_())
            del fb
        if not args.no_env:
            fb = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
            line["environment_map"] = bench_env(device, args.steps, args.warmup, lambda: fb.zero_())
            del fb
        if not args.no_train:
            line["training_step"] = bench_training_step(device)
        if not args.no_large:
            import scenes
            sc_large, _ = scenes.config(4)
            line["large_scene"] = bench_large_scene(device, sc_large)
            fb = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
            line["large_scene_fwd_bwd"] = bench_large_fwd_bwd(device, sc_large, args.steps, args.warmup,
                                                              lambda: fb.zero_())
            del fb, sc_large
        if not args.no_serve:
            line["serve"] = bench_serving(device, args.serve_seconds)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile_only:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main_reference(args):
    """The oracle timed on the host cores (all of them, OpenMP): each step is
    one forward + backward of the same workload -- the whole 5M-point cloud
    when that fits the time budget, else a random sample of its points (full
    pyramid) sized so that the whole run stays within about two minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import scenes
    sc, cams = scenes.config(2)
    cam = cams[0]
    feat = sc.feat_as("bf16")
    G = scenes.upstream_grad(cam.w, cam.h, LEVELS, sc.c, 2024)
    Gf = np.concatenate([g.ravel() for g in G]).astype(np.float64)
    cores = oracle.threads(0)
    rng = np.random.default_rng(7)
    per_step_s = max(0.5, 120.0 / max(1, args.steps + args.warmup))
    probe = np.sort(rng.choice(sc.n, 500_000, replace=False))
    t0 = time.perf_counter()
    _oracle_step(oracle, sc, feat, cam, Gf, probe, 0)
    t_probe = time.perf_counter() - t0
    m = int(min(sc.n, max(10_000, probe.size * per_step_s / max(t_probe, 1e-3))))

    def step():
        idx = None if m >= sc.n else np.sort(rng.choice(sc.n, m, replace=False))
        _oracle_step(oracle, sc, feat, cam, Gf, idx, 0)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    what = "the whole 5M-point cloud" if m >= sc.n else f"{m} points drawn from the 5M-point cloud"
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (bf16 descriptors upcast)", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "single view 1920x1080: 5M points on 50 seeded surfaces, C=8 BF16, 4 layers, "
                                   "fwd+bwd; each step " + what, "points_per_step": m},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what} per step, full 1080p pyramid, FP64 C oracle on {cores} OpenMP "
                                       "threads"},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
