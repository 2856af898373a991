"""Test stand-in for the per-rank compute of a video split along t: the same
interface as ``paper_1907_02731_gb300.slab.LibSlab``, computed by the FP64
oracle on the rank's slab (own frames plus halo) on the host.  Lets the
host-side protocol (partition, all-reduce of the step sums, halo exchange)
run on CPU ranks; the library's own slab kernels are checked on the GPU."""
import numpy as np
import torch

import oracle
from paper_1907_02731_gb300.slab import slab_frames


class OracleSlab:
    def __init__(self, s, f, a, b, radii, sigmas, alpha, p):
        nf = s.shape[0]
        self.rt = radii[0]
        self.lo, self.hi = slab_frames(nf, a, b, self.rt)
        self.o0, self.o1 = a - self.lo, b - self.lo           # own frames inside the slab
        self.sp = oracle.unary(np.asarray(s[self.lo:self.hi], np.float64), p)
        self.f = np.asarray(f[self.lo:self.hi], np.float64)
        self.radii, self.sigmas, self.alpha = radii, sigmas, alpha
        self.trace = {"rayleigh": [], "residual": []}

    def start(self, x0_slab, n_iters):
        self.x = np.asarray(x0_slab, np.float64).copy()        # stored iterate, halo frames included
        own = self.x[self.o0:self.o1]
        self.shift = 0.0
        return torch.tensor([float(np.sum(own * own))], dtype=torch.float64)

    def set_norm(self, part):
        self.scale = 1.0 / np.sqrt(float(part[0]))

    def step(self, last=False):
        xh = self.scale * self.x
        y = oracle.apply_M(self.sp, self.f, xh, self.radii, self.sigmas, self.alpha)
        self.z = y[self.o0:self.o1]
        xo = xh[self.o0:self.o1]
        d = self.z - self.shift * xo
        return torch.tensor([np.sum(self.z * self.z), np.sum(xo * self.z), np.sum(xo * xo), np.sum(d * d)],
                            dtype=torch.float64)

    def finish_step(self, sums):
        zz, xz, xx, dd = (float(v) for v in sums)
        r = xz / xx
        self.trace["rayleigh"].append(r)
        self.trace["residual"].append(np.sqrt(max(dd - (r - self.shift) ** 2 * xx, 0.0) / xx))
        self.x[self.o0:self.o1] = self.z
        self.scale = 1.0 / np.sqrt(zz)
        self.shift = r

    def pack(self, side):
        fr = self.x[self.o0:self.o0 + self.rt] if side == 0 else self.x[self.o1 - self.rt:self.o1]
        return torch.from_numpy(np.ascontiguousarray(fr))

    def recv_buffer(self, side):
        n = self.o0 if side == 0 else self.x.shape[0] - self.o1
        return torch.empty((n,) + self.x.shape[1:], dtype=torch.float64)

    def unpack(self, side, buf):
        if side == 0:
            self.x[:self.o0] = buf.numpy()
        else:
            self.x[self.o1:] = buf.numpy()

    def output(self):
        return torch.from_numpy(self.scale * self.x[self.o0:self.o1])
