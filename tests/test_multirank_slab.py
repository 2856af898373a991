"""One video split along t over 2 and 3 gloo ranks on CPU.

Each rank runs the product's host-side protocol (``slab.SlabProtocol``: the
partition, the all-reduce of the four step sums, the finalize, the halo
exchange between neighbours) over the product's transport
(``slab.TorchComm`` on torch.distributed, gloo).  The per-rank compute is the
FP64 oracle on the rank's slab (``_slab_oracle.OracleSlab``), since this host
has no GPU; the library's slab kernels are checked against the oracle on the
GPU in test_gpu_slab.py.  The concatenated own frames must equal the oracle's
whole-video iteration, and every rank must hold the same trace.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SHAPE = (11, 12, 14)
RADII, SIG, ALPHA, P, K = (2, 2, 3), (1.5, 1.0, 2.0), 0.9, 0.3, 6


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _video():
    rng = np.random.default_rng(77)
    s = rng.random(SHAPE) + 0.05
    f = rng.random(SHAPE)
    x0 = rng.random(SHAPE) + 0.1
    return s, f, x0


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1907_02731_gb300.slab import SlabProtocol, TorchComm, slab_frames, split_frames
        from _slab_oracle import OracleSlab
        s, f, x0 = _video()
        a, b = split_frames(SHAPE[0], world, RADII[0])[rank]
        lo, hi = slab_frames(SHAPE[0], a, b, RADII[0])
        ops = OracleSlab(s, f, a, b, RADII, SIG, ALPHA, P)
        x = SlabProtocol(ops, TorchComm(), rank, world).run(x0[lo:hi], K)
        np.save(os.path.join(out_dir, f"x{rank}.npy"), x.numpy())
        np.save(os.path.join(out_dir, f"t{rank}.npy"),
                np.array([ops.trace["rayleigh"], ops.trace["residual"]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_video_equals_whole_video(tmp_path, world):
    import oracle
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    s, f, x0 = _video()
    ref = oracle.power_iterate(oracle.unary(s, P), f, x0, K, RADII, SIG, ALPHA)
    x = np.concatenate([np.load(tmp_path / f"x{r}.npy") for r in range(world)])
    assert x.shape == SHAPE
    np.testing.assert_allclose(x, ref["x"], rtol=1e-10, atol=1e-13)
    tr = [np.load(tmp_path / f"t{r}.npy") for r in range(world)]
    for t in tr:
        np.testing.assert_array_equal(t, tr[0])        # one all-reduce: the same sums on every rank
    np.testing.assert_allclose(tr[0][0], ref["rayleigh"], rtol=1e-11)
    np.testing.assert_allclose(tr[0][1], ref["residual"], rtol=1e-7, atol=1e-12)


def test_split_frames_partition():
    from paper_1907_02731_gb300.slab import slab_frames, split_frames
    assert split_frames(11, 3, 2) == [(0, 4), (4, 8), (8, 11)]
    assert split_frames(72, 8, 2)[-1] == (63, 72)
    assert split_frames(5, 1, 9) == [(0, 5)]
    with pytest.raises(ValueError):
        split_frames(5, 3, 2)                          # a slab would own fewer than rt frames
    assert slab_frames(11, 4, 8, 2) == (2, 10)
    assert slab_frames(11, 0, 4, 2) == (0, 6)
    assert slab_frames(11, 8, 11, 2) == (6, 11)
