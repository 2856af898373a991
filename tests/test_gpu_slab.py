"""The library's slab kernels (a video split along t) on one GPU.

Several ranks are emulated as host threads of one process, each with its own
slab context on the same GPU, running the product's ``slab.SlabProtocol``.
The transport is a thread barrier: the step sums are added on the device and
the halo frames copied between the threads' buffers, each exchange after a
device synchronisation, so no kernel ever waits on another.  The
concatenated own frames must match the oracle's whole-video iteration.
"""
import threading

import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import slab

from _helpers import TOL_F32, TOL_LOWP, oracle_power, rel_l2, to_dev

pytestmark = pytest.mark.gpu


class ThreadComm:
    """All-reduce and neighbour exchange between threads of one process."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world)
        self.slots = {}

    def _sync(self):
        import torch
        torch.cuda.synchronize()
        self.bar.wait()

    def all_reduce_sum(self, t):
        rank = threading.current_thread().rank
        self._sync()
        self.slots[("sum", rank)] = t.clone()
        self._sync()
        acc = self.slots[("sum", 0)].clone()
        for r in range(1, self.world):
            acc += self.slots[("sum", r)]
        self._sync()
        t.copy_(acc)

    def exchange(self, rank, send_lo, recv_lo, send_hi, recv_hi):
        self._sync()
        if send_lo is not None:
            self.slots[(rank, rank - 1)] = send_lo
        if send_hi is not None:
            self.slots[(rank, rank + 1)] = send_hi
        self._sync()
        if recv_lo is not None:
            recv_lo.copy_(self.slots[(rank - 1, rank)])
        if recv_hi is not None:
            recv_hi.copy_(self.slots[(rank + 1, rank)])
        self._sync()


def run_split(s, f, x0, K, world, radii, sigmas, alpha, p, storage="f32"):
    nf = s.shape[0]
    comm = ThreadComm(world)
    bounds = slab.split_frames(nf, world, radii[0])
    out, traces, errs = [None] * world, [None] * world, []

    def rank_main(rank):
        threading.current_thread().rank = rank
        try:
            a, b = bounds[rank]
            lo, hi = slab.slab_frames(nf, a, b, radii[0])
            ops = slab.LibSlab(s.shape, a, b, radii=radii, sigmas=sigmas, alpha=alpha, p=p, storage=storage)
            try:
                ops.load_features(to_dev(s[lo:hi]), to_dev(f[lo:hi]))
                x = slab.SlabProtocol(ops, comm, rank, world).run(to_dev(x0[lo:hi]), K)
                assert ops.status() == sf.SFSEG_OK
                out[rank] = x.cpu().numpy()
                traces[rank] = ops.trace()
            finally:
                ops.close()
        except BaseException as e:   # noqa: BLE001 -- reported by the main thread
            errs.append(e)
            comm.bar.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errs:
        raise errs[0]
    return np.concatenate(out), traces


CASES = [  # (shape, radii, sigmas, world): specialised radii, any-radius kernel, uneven slabs
    ((24, 40, 70), (2, 5, 5), (1.5, 3.0, 3.0), 2),
    ((24, 40, 70), (2, 5, 5), (1.5, 3.0, 3.0), 3),
    ((13, 33, 45), (2, 4, 4), (1.5, 2.5, 2.5), 4),
    ((17, 20, 30), (3, 1, 2), (2.0, 1.0, 1.5), 3),
    ((9, 16, 20), (1, 2, 2), (1.0, 1.5, 1.5), 1),
]


@pytest.mark.parametrize("shape,radii,sig,world", CASES)
def test_split_video_matches_oracle(cuda_device, shape, radii, sig, world):
    rng = np.random.default_rng(sum(shape) + world)
    s = rng.random(shape, dtype=np.float32) + 0.05
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32) + 0.1
    K = 7
    x, traces = run_split(s, f, x0, K, world, radii, sig, 0.9, 0.3)
    ref = oracle_power(f, x0, K, radii, sig, 0.9, 0.3, s=s)
    assert rel_l2(x, ref["x"]) < TOL_F32
    for tr in traces:
        np.testing.assert_array_equal(tr["rayleigh"], traces[0]["rayleigh"])   # the same sums on every rank
    np.testing.assert_allclose(traces[0]["rayleigh"], ref["rayleigh"], rtol=1e-6)
    np.testing.assert_allclose(traces[0]["residual"], ref["residual"], rtol=1e-3,
                               atol=1e-5 * ref["rayleigh"][-1])


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_split_video_low_precision_matches_oracle(cuda_device, storage):
    rng = np.random.default_rng(5)
    shape, radii, sig = (20, 36, 52), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    x, _ = run_split(f, f, f, 8, 3, radii, sig, 1.0, 0.1, storage=storage)
    ref = oracle_power(f, f, 8, radii, sig, 1.0, 0.1, storage=storage)
    assert rel_l2(x, ref["x"]) < TOL_LOWP


def test_one_slab_equals_power_iterate(cuda_device):
    """One rank owning every frame: the split path is power_iterate in steps."""
    import torch
    rng = np.random.default_rng(6)
    shape, radii, sig = (10, 48, 64), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    x, _ = run_split(f, f, f, 9, 1, radii, sig, 1.0, 0.1)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    d = to_dev(f)
    y = eng.power_iterate(d, d, d.clone(), 9)
    torch.cuda.synchronize()
    eng.close()
    assert rel_l2(x, y.cpu().numpy()) < 1e-6
