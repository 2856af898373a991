"""Benchmark of the SFSeg power iteration on GB300.

One bench step = one whole pass of the hot path on the 854x480 x 72-frame
video with the 11x11x5 Gaussian: load features (sp = S^p, storage
conversion), 50 power steps (3D-convolution form + L2 renormalisation +
Rayleigh/residual), unit-norm FP32 output.  Metric: voxel-iterations/s
(voxels x power steps / time).  Inputs are resident in HBM for `value`; the
`e2e` figure adds the pinned host->device copy of the video and the
device->host read of the result, through the public C-ABI call.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload NAME] [--storage f32|bf16|f16]
Under torchrun (N > 1) every rank runs its own seeded video (independent
problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PATH_CHOICE = "auto"
L2_FLUSH_BYTES = 256 << 20   # twice the GB300's L2
METRIC = "voxel-iterations/sec and HBM GB/s fraction at 480p vs plain FP32, rel-L2 ≤1e-3"
UNIT = "voxel-iter/s"
STORAGE_BYTES = {"f32": 4, "bf16": 2, "f16": 2}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel at the workload's full size, from one ncu capture, with a
# hash of the kernel sources the capture was taken on.  When the sources no
# longer hash to that value the kernel has changed since the capture and the
# figure is reported as null.
KERNEL_SOURCES = ("paper_1907_02731_gb300/csrc/step_fast.cu", "paper_1907_02731_gb300/csrc/sfseg_common.cuh")
DRAM_TRAFFIC_PER_LAUNCH = {
    ("video_72x480x854", "f32"): (367743744.0 + 98644736.0, "f351d46bae071de7"),
    ("video_72x480x854", "bf16"): (181751296.0 + 39703296.0, "f351d46bae071de7"),
}


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(workload: str, storage: str):
    """(bytes per launch, None) when captured on the current kernel sources,
    else (None, reason)."""
    rec = DRAM_TRAFFIC_PER_LAUNCH.get((workload, storage))
    if rec is None:
        return None, "not captured for this workload"
    if rec[1] != kernel_hash():
        return None, "kernel changed since the capture"
    return rec[0], None


def alu_flops_per_voxel(wl) -> int:
    """Algorithmic FP32 flops of one voxel-iteration (an FMA counts 2), no
    halo recompute: pre-products a = sp x, b_c = f_c a, c = sum f_c^2 a
    (1 + 2C); the separable taps of the 2 + C convolutions (Eq. 9; 3 for one
    channel); the combine (8 per channel); the four per-voxel reduction
    terms z.z, x.z, x.x and |z - r x|^2 (10)."""
    C = wl.nchan
    nconv = 3 if C == 1 else C + 2
    taps = (2 * wl.rt + 1) + (2 * wl.ry + 1) + (2 * wl.rx + 1)
    return (1 + 2 * C) + nconv * taps * 2 + 8 * C + 10


def alu_peak_tflops(sm_max_mhz=None) -> float:
    """Plain FP32 pipe peak of this GPU: SMs x 128 FP32 lanes x 2 flops x the
    maximum SM clock (nvidia-smi's clocks.max.sm, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(sm_max_mhz) if sm_max_mhz else 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: wait for its first sample so
            # that the timed region that follows is covered, then keep only the
            # samples taken from here on
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        self.after = False
        if self.proc and not self.lines:
            # a timed region shorter than the sampling period saw no sample:
            # take the first one after it (reported as such)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 1.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.after = bool(self.lines)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
               "reasons": sorted(reasons), "samples": len(sm)}
        if getattr(self, "after", False):
            out["window"] = "timed region shorter than the 50 ms sampling period: first sample after it"
        return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(times, world, device="cpu"):
    """Element-wise maximum of per-rank times over all ranks (every rank gets
    the result): the job ends when its slowest rank does."""
    import torch
    vals = torch.tensor([float(t) for t in times], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    return [float(v) for v in vals.cpu()]


def sum_over_ranks(units, world, device="cpu"):
    """Work units (voxel-iterations) processed by all ranks together."""
    import torch
    val = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(val, op=dist.ReduceOp.SUM)
    return float(val.cpu()[0])


def rank_video_index(rank):
    """Each rank draws its own seeded video (or batch): the ranks solve
    independent problems, so nothing is exchanged on the data path."""
    return int(rank)


def cpu_baseline(wl, frames=None, iters=4, min_seconds=5.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded
    sample of the workload, in the workload's unit (voxel-iterations / s):
    the video (all its frames, or the first `frames`) and `iters` power steps
    (more when that takes under `min_seconds`, so that small volumes are timed
    over a few seconds); for the batch its first video; for the
    differentiable form 8 frames, `iters` steps forward plus the oracle's
    reverse mode (the bench step there is forward + adjoint)."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import oracle
    from paper_1907_02731_gb300 import inputs
    radii = (wl.rt, wl.ry, wl.rx)
    sig = (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    if wl.name.startswith("batch"):
        nf, h, w = inputs.batch_layout()[0]
        s = inputs.make_video(nf, h, w, inputs.config_seed(inputs.BATCH_CONFIG, 0), 2)[0]
        f, what = s, f"the first video of the batch ({w}x{h}x{nf})"
    else:
        s, f = inputs.workload_features(wl.name)
        what = f"the {wl.w}x{wl.h}x{wl.nf} video"
    grad = wl.name.startswith("grad")
    nf_s = 8 if grad else s.shape[0]
    if frames is not None and not grad:
        nf_s = max(1, min(nf_s, int(frames)))
        if nf_s < s.shape[0]:
            what = f"the first {nf_s} frames of " + what
    sub = np.ascontiguousarray(s[:nf_s], dtype=np.float64)
    fsub = np.ascontiguousarray(f[..., :nf_s, :, :], dtype=np.float64)
    sp = oracle.unary(sub, wl.p)

    def run(k):
        t0 = time.perf_counter()
        if grad:
            target = (sub > 0.5).astype(np.float64)
            oracle.adjoint(sp, fsub, sub, k, radii, sig, wl.alpha, target)
        else:
            oracle.power_iterate(sp, fsub, sub, k, radii, sig, wl.alpha)
        return time.perf_counter() - t0
    dt = run(iters)
    if dt < min_seconds:   # small volumes: enough steps for a few seconds of CPU work
        iters = min(4000, max(iters + 1, int(iters * min_seconds / max(dt, 1e-4))))
        dt = run(iters)
    if grad:
        what = f"the first {nf_s} frames of " + what + ", forward + reverse mode"
    vox_iter = sub.size * iters
    return {"value": vox_iter / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{what}, {iters} FP64 power steps, explicit edge-by-edge M ({dt:.1f} s)"}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    cb = None
    # every sample is the whole video, the same frames as the cpu_baseline
    # leg of our arm; when many steps are asked for, each sample runs fewer
    # power iterations, so that the whole run stays within a few minutes
    # (about 48 full-video iterations, 2 s each on 16 cores)
    iters = max(1, min(4, 48 // max(1, args.warmup + args.steps)))
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, iters=iters)
        steps.append(cb["value"])
    vals = steps[args.warmup:]
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "impl": "reference",
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.storage),
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(wl, storage, prob=None, split=None, world=1):
    """The config object of a bench line (the workload, its sizes and how the
    timed calls treat L2)."""
    cfg = {"workload": wl.name, "frames": wl.nf, "h": wl.h, "w": wl.w,
           "kernel": f"{2 * wl.rx + 1}x{2 * wl.ry + 1}x{2 * wl.rt + 1}",
           "sigma_xy": wl.sigma_xy, "sigma_t": wl.sigma_t, "alpha": wl.alpha, "p": wl.p,
           "iters_per_step": wl.iters, "storage": storage, "x0": "f", "channels": wl.nchan,
           "l2": ("operands larger than L2 (3 volumes of %.0f MB)" % (wl.n * 4 / 1e6)
                  if 12 * wl.n * max(1, wl.nchan) >= L2_FLUSH_BYTES else
                  "operands fit in L2 (3 volumes of %.2f MB): L2 flushed by a 256 MB write before every "
                  "timed call, CUDA events around each call" % (wl.n * 4 / 1e6))}
    if prob is not None and hasattr(prob, "dims"):
        cfg.update({"frames": None, "h": None, "w": None, "videos": len(prob.dims),
                    "voxels": prob.n, "l2": "operands larger than L2 (%.0f MB per volume set)"
                    % (prob.n * 4 / 1e6)})
    if wl.name.startswith("grad"):
        cfg["step"] = "recorded forward + adjoint (checkpoints every 8)"
    if split == "t":
        cfg["split"] = ("one video split along t over %d ranks: per step an all-reduce of 4 FP64 "
                        "sums and %d halo frames to each neighbour" % (world, wl.rt))
    return cfg


def pipelined_calls(steps, stream, h2d, compute, d2h):
    """`steps` end-to-end calls as a stream of inputs, two buffer slots: call
    i's host->device copy h2d(i % 2) runs on its own stream and overlaps call
    i-1's compute(), its device->host read d2h(i % 2) runs on a third stream
    and overlaps call i+1's compute().  Every call's copies lie inside the
    returned time (ms per call, CUDA events on `stream`)."""
    import torch
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    d2h_done = [torch.cuda.Event() for _ in range(2)]
    started = [False, False]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def issue_h2d(i):
        j = i & 1
        with torch.cuda.stream(s_h2d):
            if started[j]:
                s_h2d.wait_event(comp_done[j])        # call i-2 no longer reads slot j
            h2d(j)
            h2d_done[j].record(s_h2d)

    t0.record(stream)
    s_h2d.wait_event(t0)
    issue_h2d(0)
    for i in range(steps):
        j = i & 1
        if i + 1 < steps:
            issue_h2d(i + 1)
        stream.wait_event(h2d_done[j])
        if started[j]:
            stream.wait_event(d2h_done[j])            # call i-2's result was read
        compute(j)
        comp_done[j].record(stream)
        started[j] = True
        with torch.cuda.stream(s_d2h):
            s_d2h.wait_event(comp_done[j])
            d2h(j)
            d2h_done[j].record(s_d2h)
    for j in range(2):
        if started[j]:
            stream.wait_event(d2h_done[j])
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1) / steps


def path_flags(name: str) -> int:
    """Context flags of a --path choice: 'auto' lets the library's autotuner
    time the step paths on the first call (inside the warm-up) and keep the
    fastest; the others force one path."""
    import paper_1907_02731_gb300 as sf
    return {"auto": sf.SFSEG_AUTOTUNE, "fast": 0, "generic": sf.SFSEG_GENERIC,
            "fused": sf.SFSEG_FUSED, "cluster": sf.SFSEG_CLUSTER}[name]


class SingleVideo:
    """One seeded video of a named workload (FP32 / BF16 / FP16 storage); with
    several pairwise channels (Eq. 9) S is channel 0 and x0 = S."""

    def __init__(self, wl, storage, rank, dev, sf, inputs):
        import torch
        self.wl, self.K, self.n = wl, wl.iters, wl.n
        s_np, f_np = inputs.workload_features(wl.name, rank_video_index(rank))
        self.f_np = s_np
        self.s = torch.from_numpy(s_np).to(dev)
        self.f = self.s if wl.nchan == 1 else torch.from_numpy(f_np).to(dev)
        self.x = torch.empty_like(self.s)
        flags = path_flags(PATH_CHOICE) if wl.nchan == 1 else 0
        self.eng = sf.SFSeg((wl.nf, wl.h, wl.w), radii=(wl.rt, wl.ry, wl.rx),
                            sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy), alpha=wl.alpha, p=wl.p,
                            storage=storage, nchan=wl.nchan, flags=flags)
        self.f_host = torch.from_numpy(np.ascontiguousarray(f_np)).pin_memory()
        self.out_host = torch.empty_like(self.s, device="cpu").pin_memory()
        self.f_dev = torch.empty_like(self.f)
        self.h2d = int(self.f_host.numel() * 4)
        self.d2h = int(self.out_host.numel() * 4)

    def step(self, iters):
        self.x.copy_(self.s)                                       # x0 = S
        self.eng.power_iterate(self.s, self.f, self.x, iters, out=self.x)

    def e2e_step(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        s_dev = self.f_dev if self.wl.nchan == 1 else self.f_dev[0]   # S = channel 0
        self.x.copy_(s_dev)
        self.eng.power_iterate(s_dev, self.f_dev, self.x, self.K, out=self.x)
        self.out_host.copy_(self.x, non_blocking=True)

    def e2e_pipeline(self, steps, stream):
        import torch
        if not hasattr(self, "_pipe"):
            self._pipe = {"fd": [torch.empty_like(self.f_dev) for _ in range(2)],
                          "x": [torch.empty_like(self.x) for _ in range(2)],
                          "oh": [torch.empty_like(self.out_host).pin_memory() for _ in range(2)]}
        pp = self._pipe

        def h2d(j):
            pp["fd"][j].copy_(self.f_host, non_blocking=True)

        def compute(j):
            fd, x = pp["fd"][j], pp["x"][j]
            s_dev = fd if self.wl.nchan == 1 else fd[0]
            x.copy_(s_dev)
            self.eng.power_iterate(s_dev, fd, x, self.K, out=x)

        def d2h(j):
            pp["oh"][j].copy_(pp["x"][j], non_blocking=True)

        return pipelined_calls(steps, stream, h2d, compute, d2h)

    def check(self):
        import torch
        tr = self.eng.trace()
        return {"x_norm": float(torch.linalg.vector_norm(self.x.double())),
                "rayleigh_last": float(tr["rayleigh"][-1]),
                "residual_last": float(tr["residual"][-1])}


class Batch:
    """The uneven batch: 24 seeded videos, frames U{20..120}, resolutions from
    {320x240, 480x360, 640x360, 854x480}, 9x9x5 Gaussian, all in one launch
    per power step (replayed as a CUDA graph)."""

    def __init__(self, wl, storage, rank, dev, sf, inputs):
        import torch
        self.K = wl.iters
        dims = inputs.batch_layout()
        self.dims = dims
        self.n = sum(nf * h * w for nf, h, w in dims)
        base = 100 * rank_video_index(rank)
        self.f_np = [inputs.make_video(nf, h, w, inputs.config_seed(inputs.BATCH_CONFIG, base + i), 2)[0]
                     for i, (nf, h, w) in enumerate(dims)]
        self.fs = [torch.from_numpy(a).to(dev) for a in self.f_np]
        self.xs = [torch.empty_like(t) for t in self.fs]
        self.eng = sf.SFSeg(batch_shapes=dims, radii=(wl.rt, wl.ry, wl.rx),
                            sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy), alpha=wl.alpha, p=wl.p,
                            storage=storage, flags=path_flags(PATH_CHOICE))
        self.f_host = [torch.from_numpy(a).pin_memory() for a in self.f_np]
        self.out_host = [torch.empty_like(t).pin_memory() for t in self.f_host]
        self.f_dev = [torch.empty_like(t) for t in self.fs]
        self.h2d = self.d2h = int(sum(t.numel() for t in self.f_host) * 4)

    def step(self, iters):
        for x, f in zip(self.xs, self.fs):
            x.copy_(f)
        self.eng.power_iterate_batched(self.fs, self.fs, self.xs, iters)

    def e2e_step(self):
        for fd, fh, x in zip(self.f_dev, self.f_host, self.xs):
            fd.copy_(fh, non_blocking=True)
            x.copy_(fd)
        self.eng.power_iterate_batched(self.f_dev, self.f_dev, self.xs, self.K)
        for oh, x in zip(self.out_host, self.xs):
            oh.copy_(x, non_blocking=True)

    def e2e_pipeline(self, steps, stream):
        import torch
        if not hasattr(self, "_pipe"):
            self._pipe = {"fd": [[torch.empty_like(t) for t in self.fs] for _ in range(2)],
                          "x": [[torch.empty_like(t) for t in self.xs] for _ in range(2)],
                          "oh": [[torch.empty_like(t).pin_memory() for t in self.out_host] for _ in range(2)]}
        pp = self._pipe

        def h2d(j):
            for fd, fh in zip(pp["fd"][j], self.f_host):
                fd.copy_(fh, non_blocking=True)

        def compute(j):
            for x, fd in zip(pp["x"][j], pp["fd"][j]):
                x.copy_(fd)
            self.eng.power_iterate_batched(pp["fd"][j], pp["fd"][j], pp["x"][j], self.K)

        def d2h(j):
            for oh, x in zip(pp["oh"][j], pp["x"][j]):
                oh.copy_(x, non_blocking=True)

        return pipelined_calls(steps, stream, h2d, compute, d2h)

    def check(self):
        import torch
        return {"x_norm_min": min(float(torch.linalg.vector_norm(x.double())) for x in self.xs),
                "videos": len(self.xs), "voxels": self.n}


class SplitVideo:
    """One video split along t over the ranks (strong scaling): rank r owns a
    contiguous slab of frames plus rt halo frames per side; per power step the
    ranks all-reduce four FP64 sums (NCCL) and exchange rt frames with each
    neighbour (NCCL send/recv).  One bench step = one whole call: features of
    the slab loaded, 50 steps, the own frames of the unit-norm x^K.  Every
    rank draws the same seeded video; `n` is this rank's own voxels, so the
    sum over ranks is the whole video."""

    def __init__(self, wl, storage, rank, dev, sf, inputs, world=1):
        import torch
        from paper_1907_02731_gb300 import slab
        self.wl, self.K, self.world, self.rank = wl, wl.iters, world, rank
        s_np, f_np = inputs.workload_features(wl.name, rank_video_index(0))
        if wl.nchan != 1:
            raise SystemExit("--split t: one pairwise channel")
        a, b = slab.split_frames(wl.nf, world, wl.rt)[rank]
        lo, hi = slab.slab_frames(wl.nf, a, b, wl.rt)
        self.n = (b - a) * wl.h * wl.w
        self.s = torch.from_numpy(np.ascontiguousarray(s_np[lo:hi])).to(dev)
        self.x0 = self.s
        self.eng = slab.LibSlab((wl.nf, wl.h, wl.w), a, b, radii=(wl.rt, wl.ry, wl.rx),
                                sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy), alpha=wl.alpha, p=wl.p,
                                storage=storage)
        self.comm = slab.TorchComm() if world > 1 else slab.LocalComm()
        self.proto = slab.SlabProtocol(self.eng, self.comm, rank, world)
        self.f_host = torch.from_numpy(np.ascontiguousarray(s_np[lo:hi])).pin_memory()
        self.f_dev = torch.empty_like(self.s)
        self.out_host = torch.empty((b - a, wl.h, wl.w), dtype=torch.float32).pin_memory()
        self.h2d = int(self.f_host.numel() * 4)
        self.d2h = int(self.out_host.numel() * 4)
        self.x = None

    def step(self, iters):
        self.eng.load_features(self.s, self.s)
        self.x = self.proto.run(self.x0, iters)

    def e2e_step(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.eng.load_features(self.f_dev, self.f_dev)
        x = self.proto.run(self.f_dev, self.K)
        self.out_host.copy_(x, non_blocking=True)

    def check(self):
        import torch
        tr = self.eng.trace()
        return {"own_x_sq_norm": float(torch.sum(self.x.double() ** 2)), "ranks": self.world,
                "rayleigh_last": float(tr["rayleigh"][-1])}


class Grad:
    """Differentiable form: 854x480x48, 40 recorded power steps, then the
    adjoint of L = sum(target * x^K) w.r.t. sp, f and x0 (checkpoints every 8
    steps).  One bench step = forward + backward."""

    def __init__(self, wl, storage, rank, dev, sf, inputs):
        import torch
        from paper_1907_02731_gb300.autograd import make_engine
        self.K, self.n = wl.iters, wl.n
        seed = inputs.config_seed(wl.config, rank_video_index(rank))
        f_np, mask = inputs.make_video(wl.nf, wl.h, wl.w, seed, wl.n_distractors)
        self.f_np = f_np
        self.f = torch.from_numpy(f_np).to(dev)
        self.target = torch.from_numpy(mask.astype("float32")).to(dev)
        self.x = torch.empty_like(self.f)
        self.eng = make_engine((wl.nf, wl.h, wl.w), radii=(wl.rt, wl.ry, wl.rx),
                               sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy), alpha=wl.alpha, p=wl.p)
        self.f_host = torch.from_numpy(f_np).pin_memory()
        self.out_host = torch.empty_like(self.f_host).pin_memory()
        self.f_dev = torch.empty_like(self.f)
        self.h2d = int(self.f_host.numel() * 4)
        self.d2h = 3 * self.h2d

    def step(self, iters):
        self.x.copy_(self.f)
        self.eng.power_iterate(self.f, self.f, self.x, max(iters, 1), out=self.x)
        if iters > 0:
            self.grads = self.eng.adjoint(self.target)

    def e2e_step(self):
        self.f_dev.copy_(self.f_host, non_blocking=True)
        self.x.copy_(self.f_dev)
        self.eng.power_iterate(self.f_dev, self.f_dev, self.x, self.K, out=self.x)
        gsp, gf, gx0 = self.eng.adjoint(self.target)
        for g in (gsp, gf, gx0):
            self.out_host.copy_(g, non_blocking=True)

    def check(self):
        import torch
        gsp, gf, gx0 = self.grads
        return {"grad_x0_dot_x0_rel": float((gx0.double() * self.f.double()).sum()
                                            / (gx0.norm() * self.f.norm())),
                "grad_f_norm": float(gf.norm())}


def run_ours(args, wl):
    import torch
    import paper_1907_02731_gb300 as sf
    from paper_1907_02731_gb300 import inputs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    kind = {"batch_24": Batch, "grad_48x480x854": Grad}.get(wl.name, SingleVideo)
    if args.split == "t":
        kind = SplitVideo
        prob = kind(wl, args.storage, rank, dev, sf, inputs, world)
    else:
        prob = kind(wl, args.storage, rank, dev, sf, inputs)
    K = prob.K

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        prob.step(K)
    barrier()
    prob.path_info = prob.eng.path() if hasattr(prob.eng, "path") else {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # operands that fit in L2 (the small workloads): every timed call starts
    # from a flushed L2 (a 256 MB write, outside the call's own events)
    flush = None
    if L2_FLUSH_BYTES > 12 * prob.n * max(1, wl.nchan):
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    launches0 = prob.eng.launch_count()
    with ClockSampler(local) as clk:
        if flush is None:
            ev0.record(stream)
            for _ in range(args.steps):
                prob.step(K)
            ev1.record(stream)
            barrier()
            ms = ev0.elapsed_time(ev1) / args.steps
        else:
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for a, b in evs:
                flush.zero_()
                a.record(stream)
                prob.step(K)
                b.record(stream)
            barrier()
            ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    launches = prob.eng.launch_count() - launches0
    check = prob.check()

    # dominant kernel (the fused power step): the same calls with K and 0
    # steps, CUDA events on the launching stream; the difference is K step
    # launches (plus a pointer-table write of a few bytes).  For the
    # differentiable form: the recorded forward with K and with 1 step.
    reps = max(3, args.steps // 2)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    if kind is Grad:
        def fwd(k):
            prob.x.copy_(prob.f)
            prob.eng.power_iterate(prob.f, prob.f, prob.x, k, out=prob.x)
        e[0].record(stream)
        for _ in range(reps):
            fwd(K)
        e[1].record(stream)
        for _ in range(reps):
            fwd(1)
        e[2].record(stream)
        torch.cuda.synchronize()
        step_ms = (e[0].elapsed_time(e[1]) - e[1].elapsed_time(e[2])) / reps / (K - 1)
    else:
        if flush is None:
            e[0].record(stream)
            for _ in range(reps):
                prob.step(K)
            e[1].record(stream)
            for _ in range(reps):
                prob.step(0)
            e[2].record(stream)
            torch.cuda.synchronize()
            step_ms = (e[0].elapsed_time(e[1]) - e[1].elapsed_time(e[2])) / reps / K
        else:
            tk = []
            for k in (K, 0):
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    prob.step(k)
                    b.record(stream)
                torch.cuda.synchronize()
                tk.append(sum(a.elapsed_time(b) for a, b in ev) / reps)
            step_ms = (tk[0] - tk[1]) / K

    # end to end through the public call with host buffers
    pipelined = hasattr(prob, "e2e_pipeline")
    if pipelined:
        prob.e2e_pipeline(2, stream)
        barrier()
        e2e_ms = prob.e2e_pipeline(args.steps, stream)
        barrier()
    else:
        for _ in range(2):
            prob.e2e_step()
        barrier()
        e[0].record(stream)
        for _ in range(args.steps):
            prob.e2e_step()
        e[1].record(stream)
        barrier()
        e2e_ms = e[0].elapsed_time(e[1]) / args.steps

    # the slowest rank sets the job's time; units are summed over ranks
    ms, e2e_ms, step_ms = max_over_ranks([ms, e2e_ms, step_ms], world, dev)
    job_units = sum_over_ranks(prob.n * K, world, dev)
    value = job_units / (ms / 1e3)
    if rank == 0:
        peak, peak_kind = _peaks()
        traffic, traffic_note = dram_traffic(wl.name, args.storage)
        if kind is SplitVideo or getattr(prob, "path_info", {}).get("path") not in (None, "fast"):
            traffic, traffic_note = None, "captured for the per-step specialised kernel only"
        bpv = (3 + wl.nchan) * STORAGE_BYTES[args.storage]   # read x, sp, f_1..f_C; write y
        achieved = bpv * prob.n / (step_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong" if kind is SplitVideo else "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": dict(workload_config(wl, args.storage, prob, split=args.split, world=world),
                           path=prob.path_info or ("slab steps (per-step kernels)" if kind is SplitVideo
                                                   else "recorded per-step (specialised kernel)")),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": traffic,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                         "traffic_note": traffic_note,
                         "frac_physical": (traffic / (step_ms / 1e3) / 1e9 / peak if traffic else None),
                         "algorithmic_bytes_per_launch": bpv * prob.n,
                         "peak_kind": peak_kind,
                         "kernel": "power step (fused stencil%s)" % (
                             ", any-radius kernel, %d channels" % wl.nchan if wl.nchan > 1 else ""),
                         "step_us": step_ms * 1e3, "bytes_per_voxel": bpv},
            "e2e": {"value": job_units / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": prob.h2d, "d2h_bytes_per_step": prob.d2h,
                    "ms_per_step": e2e_ms,
                    "copies": ("overlapped with the neighbouring calls' compute (2 copy streams, "
                               "double buffers)" if pipelined else "in sequence with the compute")},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
            "check": check,
        }
        # the ALU roofline: the FP32 stencil sits near the ridge; with 2-byte
        # storage the step is bound by its FP32 arithmetic, not its bytes
        clk_sum = line["clocks"] if isinstance(line["clocks"], dict) else {}
        fpv = alu_flops_per_voxel(wl)
        alu_peak = alu_peak_tflops(clk_sum.get("sm_max_mhz"))
        alu_ach = fpv * prob.n / (step_ms / 1e3) / 1e12
        alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
               "frac": alu_ach / alu_peak, "traffic": None, "flops_per_voxel": fpv,
               "peak_kind": "derived: SMs x 128 FP32 lanes x 2 x max SM clock",
               "step_us": step_ms * 1e3}
        if args.storage == "f32":
            line["roofline_alu"] = alu
        else:
            line["roofline_hbm"] = line["roofline"]
            alu["traffic"] = line["roofline_hbm"]["traffic"]
            line["roofline"] = alu
        if args.cpu_baseline and world == 1 and kind is SingleVideo:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line))
    prob.eng.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_accuracy(args):
    """Relative L2 and max-abs error of x^K (854x480x72, 50 steps) for FP32,
    BF16 and FP16 storage against the FP64 oracle: on the same rounded
    operands (kernel error) and on the FP32 operands (total error)."""
    import numpy as np
    import torch
    import oracle
    import paper_1907_02731_gb300 as sf
    from paper_1907_02731_gb300 import inputs
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    wl = inputs.WORKLOADS["video_72x480x854"]
    f, _ = inputs.workload_video(wl.name)
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    sp32 = (f.astype(np.float32) ** np.float32(wl.p)).astype(np.float32)
    refs, out = {}, {}
    t0 = time.perf_counter()
    for st in ("f32", "bf16", "f16"):
        spr = oracle.to_storage(sp32, st).astype(np.float32)
        fr = oracle.to_storage(f, st).astype(np.float32)
        eng = sf.SFSeg(f.shape, radii=radii, sigmas=sig, alpha=wl.alpha, p=wl.p, storage=st,
                       flags=sf.SFSEG_S_IS_SP)
        d_sp, d_f = torch.from_numpy(spr).cuda(), torch.from_numpy(fr).cuda()
        x = eng.power_iterate(d_sp, d_f, d_f.clone(), wl.iters).cpu().numpy().astype(np.float64)
        eng.close()
        refs[st] = oracle.power_iterate(spr, fr, fr, wl.iters, radii, sig, wl.alpha)["x"]
        def err(a, b):
            return {"rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                    "max_abs": float(np.abs(a - b).max()), "max_ref": float(np.abs(b).max())}
        out[st] = {"vs_oracle_same_operands": err(x, refs[st]),
                   "vs_oracle_f32_operands": err(x, refs["f32"])}
    print(json.dumps({"accuracy": out, "workload": wl.name, "iters": wl.iters,
                      "oracle_seconds": time.perf_counter() - t0,
                      "oracle_threads": int(os.environ["OMP_NUM_THREADS"])}))


SWEEP_SHAPES = ((10, 20, 20), (10, 60, 107), (20, 120, 214), (36, 240, 427), (72, 480, 854))


# Largest graphs whose explicit Eq. 2 matrix the sweep builds: on the GPU
# (cuSPARSE through torch; ~300 M stored entries at 513,600 nodes) and on the
# host (scipy; ~39 M entries at 64,200 nodes).  The full video's matrix would
# hold ~1.8e10 entries.
SPARSE_GPU_MAX_NODES = 600_000
SPARSE_CPU_MAX_NODES = 100_000


def explicit_eq2_matrix(sp, f, radii, sigmas, alpha):
    """The N x N matrix of Eq. 2 built explicitly (the comparison of Fig. 2:
    power iteration on a stored sparse adjacency): one diagonal band per
    offset (dt, dy, dx) of the Gaussian box, M_ij = sp_i sp_j (1 - alpha
    (f_i - f_j)^2) g_t g_y g_x, zero outside the volume.  sp, f: FP32 torch
    tensors [nf, h, w] on the device that builds it; returns torch CSR."""
    import torch
    nf, h, w = sp.shape
    dev = sp.device
    idx = torch.arange(nf * h * w, device=dev, dtype=torch.int64).reshape(nf, h, w)
    taps = [[math.exp(-d * d / (2.0 * s * s)) for d in range(-r, r + 1)] for r, s in zip(radii, sigmas)]

    def cut(d, n):   # (source, neighbour) index ranges along one axis for offset d
        return slice(max(0, -d), n - max(0, d)), slice(max(0, d), n - max(0, -d))
    rows, cols, vals = [], [], []
    rt, ry, rx = radii
    for dt in range(-rt, rt + 1):
        ti, tj = cut(dt, nf)
        for dy in range(-ry, ry + 1):
            yi, yj = cut(dy, h)
            for dx in range(-rx, rx + 1):
                xi, xj = cut(dx, w)
                if ti.start >= ti.stop or yi.start >= yi.stop or xi.start >= xi.stop:
                    continue
                d = f[ti, yi, xi] - f[tj, yj, xj]
                g = taps[0][dt + rt] * taps[1][dy + ry] * taps[2][dx + rx]
                vals.append((sp[ti, yi, xi] * sp[tj, yj, xj] * (1.0 - alpha * d * d) * g).reshape(-1))
                rows.append(idx[ti, yi, xi].reshape(-1))
                cols.append(idx[tj, yj, xj].reshape(-1))
    n = nf * h * w
    ij = torch.stack([torch.cat(rows), torch.cat(cols)])
    del rows, cols
    A = torch.sparse_coo_tensor(ij, torch.cat(vals), (n, n), check_invariants=False).coalesce().to_sparse_csr()
    return A


def sparse_baselines(f, sp, wl, iters, x_ours):
    """Fig. 2's comparison at one size: build the explicit matrix and run
    `iters` power steps on it (GPU: torch CSR / cuSPARSE; host: scipy), and
    the host Lanczos (scipy eigsh) for the leading eigenvector.  Times in
    seconds; x^iters of the GPU sparse run is checked against ours."""
    import torch
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    n = f.numel()
    out = {"sparse_gpu": None, "sparse_cpu": None, "lanczos_cpu": None}
    if n <= SPARSE_GPU_MAX_NODES:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A = explicit_eq2_matrix(sp, f, radii, sig, wl.alpha)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        x = f.reshape(-1) / f.norm()
        for _ in range(3):   # warm-up of the SpMV path
            y = A @ x
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        for _ in range(iters):
            y = A @ x
            x = y / y.norm()
        e[1].record()
        torch.cuda.synchronize()
        err = float((x - x_ours.reshape(-1)).norm() / x_ours.norm())
        out["sparse_gpu"] = {"build_s": t_build, "iters_s": e[0].elapsed_time(e[1]) / 1e3,
                             "nnz": int(A.values().numel()), "rel_l2_vs_ours": err}
        del A, x, y
        torch.cuda.empty_cache()
    if n <= SPARSE_CPU_MAX_NODES:
        import scipy.sparse as ssp
        import scipy.sparse.linalg as sla
        fc, spc = f.cpu(), sp.cpu()
        t0 = time.perf_counter()
        Ac = explicit_eq2_matrix(spc, fc, radii, sig, wl.alpha)
        A = ssp.csr_matrix((Ac.values().numpy(), Ac.col_indices().numpy(), Ac.crow_indices().numpy()),
                           shape=(n, n))
        t_build = time.perf_counter() - t0
        x = fc.reshape(-1).numpy().astype(np.float32)
        x /= np.linalg.norm(x)
        t0 = time.perf_counter()
        for _ in range(iters):
            y = A @ x
            x = y / np.linalg.norm(y)
        t_it = time.perf_counter() - t0
        out["sparse_cpu"] = {"build_s": t_build, "iters_s": t_it, "threads": 1}
        t0 = time.perf_counter()
        sla.eigsh(A.astype(np.float64), k=1, which="LA", tol=1e-8)
        out["lanczos_cpu"] = {"eigsh_s": time.perf_counter() - t0}
    return out


def run_sweep(args):
    """Runtime of one power step against the number of nodes (Fig. 2): the
    same 11x11x5 kernel and seeded video recipe from the paper's 4000-node toy
    to the full 854x480x72 video; one JSON line per size.  With --sweep-sparse
    the line adds Fig. 2's comparison: 100 power steps on the explicitly built
    sparse matrix (GPU and host) and host Lanczos, up to the sizes whose
    matrix is practical to store."""
    import torch
    import paper_1907_02731_gb300 as sf
    from paper_1907_02731_gb300 import inputs
    wl = inputs.WORKLOADS["video_72x480x854"]
    if args.sweep_sparse:   # torch's sparse set-up and cuSPARSE handles, outside the timings
        t = torch.rand(2, 4, 4, device="cuda")
        _ = explicit_eq2_matrix(t, t, (1, 1, 1), (1.0, 1.0, 1.0), 1.0) @ t.reshape(-1)
        torch.cuda.synchronize()
    for shape in SWEEP_SHAPES:
        f_np, _ = inputs.make_video(*shape, inputs.config_seed(wl.config, 0), wl.n_distractors)
        f = torch.from_numpy(f_np).cuda()
        x = torch.empty_like(f)
        eng = sf.SFSeg(shape, radii=(wl.rt, wl.ry, wl.rx), sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy),
                       alpha=wl.alpha, p=wl.p, storage=args.storage,
                       flags=args.sweep_flags or path_flags(args.path))

        def call(k):
            x.copy_(f)
            eng.power_iterate(f, f, x, k, out=x)
        for _ in range(max(args.warmup, 3)):
            call(wl.iters)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        reps = max(args.steps, 5)
        e[0].record()
        for _ in range(reps):
            call(wl.iters)
        e[1].record()
        for _ in range(reps):
            call(0)
        e[2].record()
        torch.cuda.synchronize()
        step_ms = (e[0].elapsed_time(e[1]) - e[1].elapsed_time(e[2])) / reps / wl.iters
        n = int(np.prod(shape))
        line = {"sweep": "power step vs nodes", "shape": list(shape), "nodes": n,
                "storage": args.storage, "flags": args.sweep_flags, "path": eng.path(),
                "l2": "not flushed between calls (a call's steps reuse its operands from L2 anyway)",
                "us_per_step": step_ms * 1e3,
                "voxel_iter_per_s": n / (step_ms / 1e3),
                "call_ms_50_steps": e[0].elapsed_time(e[1]) / reps}
        if args.sweep_sparse:
            # Fig. 2 counts 100 iterations including the set-up: one call of
            # 100 steps (feature preparation included) against the explicit
            # matrix's build plus 100 sparse power steps
            x.copy_(f)
            torch.cuda.synchronize()
            e[0].record()
            eng.power_iterate(f, f, x, 100, out=x)
            e[1].record()
            torch.cuda.synchronize()
            line["ours_100_iters_s"] = e[0].elapsed_time(e[1]) / 1e3
            sp = f.clamp_min(0) ** wl.p if wl.p != 1.0 else f
            line.update(sparse_baselines(f, sp, wl, 100, x))
        print(json.dumps(line), flush=True)
        eng.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="video_72x480x854")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--path", default="auto", choices=["auto", "fast", "generic", "fused", "cluster"],
                    help="step path of the power iteration (auto: the library's autotuner)")
    ap.add_argument("--split", default=None, choices=["t"],
                    help="one video split along t over the ranks (strong scaling) instead of one "
                         "video per rank")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--accuracy", action="store_true",
                    help="report x^K errors of FP32/BF16/FP16 storage against the FP64 oracle")
    ap.add_argument("--sweep", action="store_true",
                    help="time one power step at sizes from 4000 nodes to the full video")
    ap.add_argument("--sweep-sparse", action="store_true",
                    help="with --sweep: also time the explicit sparse matrix (GPU, host) and host Lanczos")
    ap.add_argument("--sweep-flags", type=int, default=0,
                    help="context flags for --sweep (8: force the any-radius kernel)")
    args = ap.parse_args()
    global PATH_CHOICE
    PATH_CHOICE = args.path
    if args.sweep:
        run_sweep(args)
        return
    from paper_1907_02731_gb300 import inputs
    if args.accuracy:
        run_accuracy(args)
        return
    wl = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
