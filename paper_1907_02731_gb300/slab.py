"""One video split along t over several ranks (one process per GPU).

The power step of Eq. 7 is a local stencil (a separable Gaussian of radii
(rt, ry, rx)); Sec. 4 calls the method highly parallelisable.  A video of nf
frames is cut into contiguous slabs of frames, rank r owning [a_r, b_r) and
keeping up to rt halo frames on each side.  Per power step every rank

  1. computes y = M x on its own frames (``sfseg_slab_step``), which yields the
     four FP64 sums of its frames (z.z, x.z, x.x, |z - s x|^2);
  2. sums them over all ranks (one all-reduce of 4 doubles);
  3. applies the global sums (``sfseg_slab_finish_step``): norm, Rayleigh
     quotient, residual and the next scale, the same on every rank (Eq. 3,
     Eq. 8);
  4. exchanges rt frames of the new stored iterate with each neighbour.

``SlabProtocol`` is that sequence for one rank, written against two small
interfaces: the per-rank compute (``LibSlab``: the C-ABI library on this
rank's GPU) and the transport (``TorchComm``: torch.distributed, NCCL for
CUDA tensors, gloo for host tensors).  The module does no arithmetic of the
method: every step of the path runs in the library's kernels; torch only
carries bytes and sums four doubles per step.
"""
from __future__ import annotations

from . import (SFSEG_OK, _dev_f32, _stream_handle, sfseg_create_slab, sfseg_default_params,
               sfseg_destroy, sfseg_get_trace, sfseg_launch_count, sfseg_load_features,
               sfseg_slab_finish_step,
               sfseg_slab_halo, sfseg_slab_halo_bytes, sfseg_slab_output, sfseg_slab_set_norm,
               sfseg_slab_start, sfseg_slab_step, sfseg_sync_status, STORAGE)


def split_frames(nf: int, world: int, rt: int):
    """Contiguous near-equal frame ranges [a_r, b_r) of the ranks.  With more
    than one rank every slab must own at least rt frames (then each halo comes
    from one neighbour); ValueError otherwise."""
    if world < 1 or nf < 1:
        raise ValueError("world and nf must be >= 1")
    base, extra = divmod(nf, world)
    bounds, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        bounds.append((a, b))
        a = b
    if world > 1 and min(b - a for a, b in bounds) < max(rt, 1):
        raise ValueError(f"{nf} frames over {world} ranks: a slab owns fewer than rt = {rt} frames")
    return bounds


def slab_frames(nf: int, a: int, b: int, rt: int):
    """The frames [lo, hi) a rank owning [a, b) keeps: its own plus the halo."""
    return max(0, a - rt), min(nf, b + rt)


class SlabProtocol:
    """The host-side sequence of one rank (start, then per step: compute, sum
    over ranks, finalize, halo exchange).  ``ops`` computes, ``comm`` moves."""

    def __init__(self, ops, comm, rank: int, world: int):
        self.ops, self.comm, self.rank, self.world = ops, comm, rank, world

    def exchange(self):
        lo = self.rank > 0               # a neighbour owns the frames below
        hi = self.rank < self.world - 1  # ... and above
        send_lo = self.ops.pack(0) if lo else None
        send_hi = self.ops.pack(1) if hi else None
        recv_lo = self.ops.recv_buffer(0) if lo else None
        recv_hi = self.ops.recv_buffer(1) if hi else None
        self.comm.exchange(self.rank, send_lo, recv_lo, send_hi, recv_hi)
        if lo:
            self.ops.unpack(0, recv_lo)
        if hi:
            self.ops.unpack(1, recv_hi)

    def run(self, x0_slab, n_iters: int):
        part = self.ops.start(x0_slab, n_iters)
        self.comm.all_reduce_sum(part)
        self.ops.set_norm(part)
        for k in range(n_iters):
            last = k == n_iters - 1
            sums = self.ops.step(last)
            self.comm.all_reduce_sum(sums)
            self.ops.finish_step(sums)
            if not last:              # the halo of the output is never read
                self.exchange()
        return self.ops.output()


class LocalComm:
    """The transport of a single rank: nothing to sum with, no neighbours."""

    def all_reduce_sum(self, t):
        pass

    def exchange(self, rank, send_lo, recv_lo, send_hi, recv_hi):
        pass


class TorchComm:
    """Transport over torch.distributed (an initialised default group):
    all-reduce of the step sums, and send/recv of halo frames between
    neighbouring ranks."""

    def all_reduce_sum(self, t):
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)

    def exchange(self, rank, send_lo, recv_lo, send_hi, recv_hi):
        import torch.distributed as dist
        ops = []
        if send_lo is not None:
            ops += [dist.P2POp(dist.isend, send_lo, rank - 1), dist.P2POp(dist.irecv, recv_lo, rank - 1)]
        if send_hi is not None:
            ops += [dist.P2POp(dist.isend, send_hi, rank + 1), dist.P2POp(dist.irecv, recv_hi, rank + 1)]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


class LibSlab:
    """This rank's slab on its GPU through the C-ABI: the context over the
    slab's frames (own frames [a, b) of an nf-frame video), the device words
    of the step sums and the halo buffers (uint8 tensors on the device)."""

    def __init__(self, video_shape, a: int, b: int, *, radii=(2, 5, 5), sigmas=(1.5, 3.0, 3.0),
                 alpha=1.0, p=0.1, storage="f32", flags=0):
        import torch
        nf, h, w = video_shape
        rt = radii[0]
        self.lo, self.hi = slab_frames(nf, a, b, rt)
        self.a, self.b = a, b
        prm = sfseg_default_params(self.hi - self.lo, h, w)
        prm.rt, prm.ry, prm.rx = radii
        prm.sigma_t, prm.sigma_y, prm.sigma_x = sigmas
        prm.alpha, prm.p = alpha, p
        prm.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        prm.flags = flags
        self.ctx = sfseg_create_slab(prm, a - self.lo, b - self.lo, nf * h * w)
        self.shape = (self.hi - self.lo, h, w)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.part1 = torch.zeros(1, dtype=torch.float64, device=dev)
        self.part4 = torch.zeros(4, dtype=torch.float64, device=dev)
        self.bufs = {}
        self.final = None
        for side in (0, 1):
            for d in (0, 1):
                n = sfseg_slab_halo_bytes(self.ctx, side, d)
                self.bufs[(side, d)] = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)[:n]

    def close(self):
        if getattr(self, "ctx", None):
            sfseg_destroy(self.ctx)
            self.ctx = None

    def load_features(self, s_slab, f_slab):
        sfseg_load_features(self.ctx, _dev_f32(s_slab, "s").data_ptr(), _dev_f32(f_slab, "f").data_ptr(),
                            _stream_handle())

    def start(self, x0_slab, n_iters):
        sfseg_slab_start(self.ctx, _dev_f32(x0_slab, "x0").data_ptr(), n_iters, self.part1.data_ptr(),
                         _stream_handle())
        return self.part1

    def set_norm(self, part):
        sfseg_slab_set_norm(self.ctx, part.data_ptr(), _stream_handle())

    def step(self, last=False):
        """One step; the last one writes its output in FP32 (own frames)."""
        import torch
        final = None
        if last:
            nf, h, w = self.shape
            self.final = torch.empty((self.b - self.a, h, w), dtype=torch.float32, device=self.part1.device)
            final = self.final.data_ptr()
        sfseg_slab_step(self.ctx, self.part4.data_ptr(), final, _stream_handle())
        return self.part4

    def finish_step(self, sums):
        sfseg_slab_finish_step(self.ctx, sums.data_ptr(), _stream_handle())

    def pack(self, side):
        buf = self.bufs[(side, 0)]
        if buf.numel():
            sfseg_slab_halo(self.ctx, side, 0, buf.data_ptr(), _stream_handle())
        return buf

    def recv_buffer(self, side):
        return self.bufs[(side, 1)]

    def unpack(self, side, buf):
        if buf.numel():
            sfseg_slab_halo(self.ctx, side, 1, buf.data_ptr(), _stream_handle())

    def output(self):
        import torch
        nf, h, w = self.shape
        out = getattr(self, "final", None)
        if out is None:   # no step ran: x0 normalised, from the stored iterate
            out = torch.empty((self.b - self.a, h, w), dtype=torch.float32, device=self.part1.device)
        self.final = None
        sfseg_slab_output(self.ctx, out.data_ptr(), _stream_handle())
        return out

    def trace(self):
        return sfseg_get_trace(self.ctx, 0)

    def launch_count(self) -> int:
        return sfseg_launch_count(self.ctx)

    def status(self) -> int:
        return sfseg_sync_status(self.ctx)


def power_iterate_split(s_slab, f_slab, x0_slab, n_iters: int, video_shape, rank: int, world: int,
                        comm=None, **kw):
    """This rank's own frames of x^K for a video split along t over `world`
    ranks (the default process group; s/f/x0 are the rank's slab frames, halo
    included, as CUDA tensors).  Returns (x_own, trace, status)."""
    nf = video_shape[0]
    rt = kw.get("radii", (2, 5, 5))[0]
    a, b = split_frames(nf, world, rt)[rank]
    ops = LibSlab(video_shape, a, b, **kw)
    try:
        ops.load_features(s_slab, f_slab)
        comm = comm or (TorchComm() if world > 1 else LocalComm())
        x = SlabProtocol(ops, comm, rank, world).run(x0_slab, n_iters)
        st = ops.status()
        return x, ops.trace(), st
    finally:
        ops.close()


__all__ = ["split_frames", "slab_frames", "SlabProtocol", "LocalComm", "TorchComm", "LibSlab",
           "power_iterate_split",
           "SFSEG_OK"]
