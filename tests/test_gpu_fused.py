"""The fused path (all K power steps in one cooperative launch) and the
autotuner that chooses between step paths, against the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs

from _helpers import TOL_F32, TOL_LOWP, gpu_power, oracle_power, rel_l2, to_dev

pytestmark = pytest.mark.gpu

FUSED = sf.SFSEG_FUSED


def test_fused_small_workload_matches_oracle(cuda_device):
    """16x64x64, 7x7x7 Gaussian, 30 steps from x0 = f, in one launch."""
    wl = inputs.WORKLOADS["small_16x64x64"]
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    f, _ = inputs.workload_video(wl.name)
    x, tr, st, n = gpu_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p, flags=FUSED)
    ref = oracle_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p)
    assert st == sf.SFSEG_OK and n == wl.iters
    assert rel_l2(x, ref["x"]) < TOL_F32
    assert abs(np.linalg.norm(x) - 1) < 1e-6
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    np.testing.assert_allclose(tr["norms"], ref["norms"], rtol=1e-6)
    np.testing.assert_allclose(tr["residual"], ref["residual"], rtol=1e-3,
                               atol=1e-5 * ref["rayleigh"][-1])
    assert np.all(x >= -1e-7)


ODD = [  # ragged 32x16 tiles, shapes smaller than the kernel, one frame, one voxel
    ((1, 1, 1), (2, 5, 5), (1.5, 3.0, 3.0)),
    ((1, 5, 7), (0, 2, 3), (1.0, 1.0, 2.0)),
    ((3, 17, 33), (1, 5, 5), (1.5, 3.0, 3.0)),
    ((5, 40, 70), (2, 4, 4), (1.5, 2.5, 2.5)),
    ((2, 3, 100), (3, 1, 7), (2.0, 0.8, 4.0)),
    ((9, 1, 50), (4, 0, 2), (1.2, 1.0, 1.1)),
    ((4, 33, 65), (2, 16, 16), (1.5, 6.0, 6.0)),
    ((20, 18, 9), (8, 3, 1), (3.0, 2.0, 1.0)),
    ((7, 130, 1100), (2, 5, 5), (1.5, 3.0, 3.0)),   # rows of one voxel per phase-2 unit
]


@pytest.mark.parametrize("shape,radii,sig", ODD)
def test_fused_odd_shapes_match_oracle(cuda_device, shape, radii, sig):
    rng = np.random.default_rng(sum(shape) + 7 * sum(radii))
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32) + 0.1
    K = 4 if np.prod(shape) < 500_000 else 2
    x, tr, st, _ = gpu_power(f, x0, K, radii, sig, 0.8, 0.3, flags=FUSED)
    ref = oracle_power(f, x0, K, radii, sig, 0.8, 0.3)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_fused_low_precision_storage(cuda_device, storage):
    rng = np.random.default_rng(21)
    shape, radii, sig = (6, 40, 52), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    x, _, st, _ = gpu_power(f, f, 12, radii, sig, 1.0, 0.1, storage=storage, flags=FUSED)
    ref = oracle_power(f, f, 12, radii, sig, 1.0, 0.1, storage=storage)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_LOWP


def test_fused_batched_matches_oracle(cuda_device):
    """Uneven videos: every phase-2 range may span several videos."""
    import torch
    shapes = [(5, 24, 40), (9, 31, 17), (3, 40, 64), (1, 7, 9), (12, 20, 20)]
    rng = np.random.default_rng(10)
    fs = [rng.random(s, dtype=np.float32) for s in shapes]
    radii, sig = (2, 4, 4), (1.5, 2.5, 2.5)
    eng = sf.SFSeg(batch_shapes=shapes, radii=radii, sigmas=sig, alpha=1.0, p=0.1, flags=FUSED)
    xs = [to_dev(f) for f in fs]
    eng.power_iterate_batched([to_dev(f) for f in fs], [to_dev(f) for f in fs], xs, 7)
    torch.cuda.synchronize()
    traces = [eng.trace(v) for v in range(len(shapes))]
    assert eng.path()["path"] == "fused"
    eng.close()
    for f, xb, tb in zip(fs, xs, traces):
        ref = oracle_power(f, f, 7, radii, sig, 1.0, 0.1)
        assert rel_l2(xb.cpu().numpy(), ref["x"]) < TOL_F32
        np.testing.assert_allclose(tb["rayleigh"], ref["rayleigh"], rtol=1e-6)


def test_fused_early_stop_and_zero_norm(cuda_device):
    rng = np.random.default_rng(8)
    shape, radii, sig = (4, 8, 8), (1, 2, 2), (1.0, 1.5, 1.5)
    f = rng.random(shape, dtype=np.float32)
    x, tr, st, done = gpu_power(f, f, 3000, radii, sig, 1.0, 0.1, tol=1e-4, flags=FUSED)
    assert st == sf.SFSEG_OK and 0 < done < 3000
    assert tr["residual"][-1] < 1e-4 * tr["rayleigh"][-1]
    assert tr["residual"][-2] >= 1e-4 * tr["rayleigh"][-2]
    ref = oracle.power_iterate(oracle.unary(f, 0.1), f, f, done, radii, sig, 1.0)
    assert rel_l2(x, ref["x"]) < TOL_F32
    # x0 supported where sp = 0 only: ||M x0|| = 0 at step 0
    s = np.ones((2, 8, 8), np.float32)
    s[0, 0, 0] = 0.0
    x0 = np.zeros((2, 8, 8), np.float32)
    x0[0, 0, 0] = 3.0
    x, _, st, done = gpu_power(np.zeros((2, 8, 8), np.float32), x0, 5, (1, 1, 1), (1, 1, 1), 1.0,
                               1.0, s=s, tol=1e-9, flags=FUSED)
    assert st == sf.SFSEG_EZERONORM and done == 0
    assert x[0, 0, 0] == 1.0 and np.count_nonzero(x) == 1


def test_fused_is_deterministic_and_reusable(cuda_device):
    import torch
    rng = np.random.default_rng(12)
    shape = (10, 60, 107)
    f = to_dev(rng.random(shape, dtype=np.float32))
    eng = sf.SFSeg(shape, radii=(2, 5, 5), sigmas=(1.5, 3.0, 3.0), flags=FUSED)
    try:
        a = eng.power_iterate(f, f, f.clone(), 20)
        b = eng.power_iterate(f, f, f.clone(), 20)
        c = eng.power_iterate(f, f, f.clone(), 5)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        ref = oracle.power_iterate(oracle.unary(f.cpu().numpy(), 0.1), f.cpu().numpy(),
                                   f.cpu().numpy(), 5, (2, 5, 5), (1.5, 3.0, 3.0), 1.0)
        assert rel_l2(c.cpu().numpy(), ref["x"]) < TOL_F32
    finally:
        eng.close()


def test_fused_barrier_timeout_is_reported_and_recovers(cuda_device):
    """CTA 0 waits at the first grid barrier without arriving (a barrier that
    can never complete): every CTA gives up after the 1 s limit, the call
    reports SFSEG_ETIMEOUT, and the context computes correctly afterwards."""
    import torch
    rng = np.random.default_rng(13)
    shape = (8, 40, 60)
    f = to_dev(rng.random(shape, dtype=np.float32))
    eng = sf.SFSeg(shape, radii=(2, 4, 4), sigmas=(1.5, 2.5, 2.5), flags=FUSED)
    try:
        ref = eng.power_iterate(f, f, f.clone(), 6)
        assert eng.sync_status() == sf.SFSEG_OK
        eng.debug_inject_timeout(1)
        t0 = time.time()
        x = eng.power_iterate(f, f, f.clone(), 6)
        st = eng.sync_status()
        dt = time.time() - t0
        assert st == sf.SFSEG_ETIMEOUT
        assert dt < 10.0
        assert torch.isfinite(x).all()
        again = eng.power_iterate(f, f, f.clone(), 6)
        assert eng.sync_status() == sf.SFSEG_OK
        assert torch.equal(again, ref)
    finally:
        eng.close()


def test_autotune_choice_matches_oracle_and_is_cached(cuda_device):
    """The autotuner times the per-step kernel, the fused launch and the
    cluster launch on the context's own inputs; whichever it keeps, the result
    is the oracle's."""
    import torch
    wl = inputs.WORKLOADS["small_16x64x64"]
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    f, _ = inputs.workload_video(wl.name)
    eng = sf.SFSeg(f.shape, radii=radii, sigmas=sig, alpha=wl.alpha, p=wl.p, flags=sf.SFSEG_AUTOTUNE)
    try:
        d = to_dev(f)
        x = eng.power_iterate(d, d, d.clone(), wl.iters)
        torch.cuda.synchronize()
        info = eng.path()
        assert info["path"] in ("generic", "fused", "cluster")   # 7x7x7 has no specialised kernel
        assert set(info["tuned_us"]) == {"generic", "fused", "cluster"}
        assert all(u > 0 for u in info["tuned_us"].values())
        best = min(info["tuned_us"], key=info["tuned_us"].get)
        assert info["path"] == best
        ref = oracle_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p)
        assert rel_l2(x.cpu().numpy(), ref["x"]) < TOL_F32
        tr = eng.trace()
        np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    finally:
        eng.close()
    eng2 = sf.SFSeg(f.shape, radii=radii, sigmas=sig, alpha=wl.alpha, p=wl.p, flags=sf.SFSEG_AUTOTUNE)
    try:
        d = to_dev(f)
        eng2.power_iterate(d, d, d.clone(), 3)
        assert eng2.path() == info                          # same shape class: the cached choice
    finally:
        eng2.close()


def test_autotune_batched_matches_oracle(cuda_device):
    """A batch of small uneven videos on the specialised radii: the autotuner
    chooses among all three paths; every video equals the oracle."""
    import torch
    shapes = [(6, 30, 44), (4, 17, 90), (9, 40, 40)]
    rng = np.random.default_rng(14)
    fs = [rng.random(s, dtype=np.float32) for s in shapes]
    radii, sig = (2, 5, 5), (1.5, 3.0, 3.0)
    eng = sf.SFSeg(batch_shapes=shapes, radii=radii, sigmas=sig, alpha=1.0, p=0.1,
                   flags=sf.SFSEG_AUTOTUNE)
    xs = [to_dev(f) for f in fs]
    eng.power_iterate_batched([to_dev(f) for f in fs], [to_dev(f) for f in fs], xs, 8)
    torch.cuda.synchronize()
    info = eng.path()
    eng.close()
    assert set(info["tuned_us"]) == {"fast", "generic", "fused"}
    assert info["path"] == min(info["tuned_us"], key=info["tuned_us"].get)
    for f, xb in zip(fs, xs):
        ref = oracle_power(f, f, 8, radii, sig, 1.0, 0.1)
        assert rel_l2(xb.cpu().numpy(), ref["x"]) < TOL_F32


def test_autotuned_context_serves_every_entry_point(cuda_device):
    """After the autotuner kept the fused or cluster launch, the per-step entry points of
    the same context (Rayleigh quotient, one application of M, the binarised
    iteration) still run their one-launch-per-step kernels and match the
    oracle."""
    import torch
    from oracle import binarize
    rng = np.random.default_rng(15)
    shape, radii, sig = (6, 24, 40), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=1.0, p=0.1, flags=sf.SFSEG_AUTOTUNE)
    try:
        d = to_dev(f)
        x = eng.power_iterate(d, d, d.clone(), 10)
        torch.cuda.synchronize()
        assert eng.path()["path"] in ("fast", "fused", "cluster")
        ref = oracle_power(f, f, 10, radii, sig, 1.0, 0.1)
        assert rel_l2(x.cpu().numpy(), ref["x"]) < TOL_F32
        xv = rng.standard_normal(shape).astype(np.float32)
        y = eng.apply(to_dev(xv)).cpu().numpy()
        sp = oracle.unary(f, 0.1)
        assert rel_l2(y, oracle.apply_M(sp, f, xv, radii, sig, 1.0)) < 1e-6
        lam, _ = eng.rayleigh(to_dev(f))
        r1 = oracle.power_iterate(sp, f, f, 1, radii, sig, 1.0)
        assert abs(lam - r1["rayleigh"][0]) < 1e-6 * abs(r1["rayleigh"][0])
        xb, mask = eng.power_iterate_binarized(d, d, d.clone(), 6, k0=3)
        rb = binarize.power_iterate_binarized(sp, f, f, 6, radii, sig, 1.0, 3, 10.0, 0.5, 0.5)
        assert rel_l2(xb.cpu().numpy(), rb["x"]) < 1e-5 * 2.5 ** 3
    finally:
        eng.close()
