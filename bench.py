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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/sec and HBM GB/s fraction at 480p vs plain FP32, rel-L2 ≤1e-3"
UNIT = "voxel-iter/s"
STORAGE_BYTES = {"f32": 4, "bf16": 2, "f16": 2}


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(wl, seconds_hint: float = 15.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded
    sample of the workload: the first `nf_s` frames of the same video and a
    few power steps."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import numpy as np
    import oracle
    from paper_1907_02731_gb300 import inputs
    f, _ = inputs.workload_video(wl.name)
    nf_s, iters = wl.nf, 4
    sub = np.ascontiguousarray(f[:nf_s], dtype=np.float64)
    radii = (wl.rt, wl.ry, wl.rx)
    sig = (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    sp = oracle.unary(sub, wl.p)
    t0 = time.perf_counter()
    oracle.power_iterate(sp, sub, sub, iters, radii, sig, wl.alpha)
    dt = time.perf_counter() - t0
    vox_iter = sub.size * iters
    return {"value": vox_iter / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"first {nf_s} of {wl.nf} frames of the {wl.w}x{wl.h} video, {iters} FP64 "
                      f"power steps, explicit edge-by-edge M ({dt:.1f} s)"}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    cb = None
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(wl)
        steps.append(cb["value"])
    vals = steps[args.warmup:]
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "impl": "reference",
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, "f64"),
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(wl, storage):
    return {"workload": wl.name, "frames": wl.nf, "h": wl.h, "w": wl.w,
            "kernel": f"{2 * wl.rx + 1}x{2 * wl.ry + 1}x{2 * wl.rt + 1}",
            "sigma_xy": wl.sigma_xy, "sigma_t": wl.sigma_t, "alpha": wl.alpha, "p": wl.p,
            "iters_per_step": wl.iters, "storage": storage, "x0": "f",
            "l2": "operands larger than L2 (3 volumes of %.0f MB)" % (wl.n * 4 / 1e6)}


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

    f_np, _ = inputs.make_video(wl.nf, wl.h, wl.w, inputs.config_seed(wl.config, rank),
                                wl.n_distractors)
    f = torch.from_numpy(f_np).to(dev)
    x = torch.empty_like(f)
    eng = sf.SFSeg((wl.nf, wl.h, wl.w), radii=(wl.rt, wl.ry, wl.rx),
                   sigmas=(wl.sigma_t, wl.sigma_xy, wl.sigma_xy), alpha=wl.alpha, p=wl.p,
                   storage=args.storage)
    K = wl.iters

    def step(iters=K):
        x.copy_(f)                                       # x0 = f
        eng.power_iterate(f, f, x, iters, out=x)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = eng.launch_count()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = eng.launch_count() - launches0
    tr = eng.trace()
    xn = float(torch.linalg.vector_norm(x.double()))

    # dominant kernel (the fused power step): the same calls with K and 0
    # steps, CUDA events on the launching stream; the difference is K step
    # launches (plus a pointer-table write of a few bytes).
    reps = max(3, args.steps // 2)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    for _ in range(reps):
        step(K)
    e[1].record(stream)
    for _ in range(reps):
        step(0)
    e[2].record(stream)
    torch.cuda.synchronize()
    t_full = e[0].elapsed_time(e[1]) / reps
    t_zero = e[1].elapsed_time(e[2]) / reps
    step_ms = (t_full - t_zero) / K

    # end to end through the public call with host buffers
    f_host = torch.from_numpy(f_np).pin_memory()
    out_host = torch.empty_like(f_host).pin_memory()
    f_dev = torch.empty_like(f)

    def e2e_step():
        f_dev.copy_(f_host, non_blocking=True)
        x.copy_(f_dev)
        eng.power_iterate(f_dev, f_dev, x, K, out=x)
        out_host.copy_(x, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    e[0].record(stream)
    for _ in range(args.steps):
        e2e_step()
    e[1].record(stream)
    barrier()
    e2e_ms = e[0].elapsed_time(e[1]) / args.steps

    # max over ranks
    vals = torch.tensor([ms, e2e_ms, step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(vals, op=torch.distributed.ReduceOp.MAX)
    ms, e2e_ms, step_ms = (float(v) for v in vals.cpu())
    vox_iter = wl.n * K
    value = world * vox_iter / (ms / 1e3)
    if rank == 0:
        peak, peak_kind = _peaks()
        bpv = 4 * STORAGE_BYTES[args.storage]          # read x, sp, f; write y
        achieved = bpv * wl.n / (step_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.storage, "data": "synthetic",
            "config": workload_config(wl, args.storage),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_kind": peak_kind, "kernel": "power step (fused stencil)",
                         "step_us": step_ms * 1e3, "bytes_per_voxel": bpv},
            "e2e": {"value": world * vox_iter / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(f_host.numel() * 4),
                    "d2h_bytes_per_step": int(out_host.numel() * 4), "ms_per_step": e2e_ms},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
            "check": {"x_norm": xn, "rayleigh_last": float(tr["rayleigh"][-1]),
                      "residual_last": float(tr["residual"][-1])},
        }
        if args.cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line))
    eng.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="video_72x480x854")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    from paper_1907_02731_gb300 import inputs
    wl = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
