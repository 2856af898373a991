"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs

from _helpers import TOL_F32, TOL_LOWP, gpu_power, oracle_power, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _wl(name):
    wl = inputs.WORKLOADS[name]
    return wl, (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)


def test_small_workload_matches_oracle(cuda_device):
    """16x64x64, 7x7x7 Gaussian, 30 steps from x0 = f (the small workload)."""
    wl, radii, sig = _wl("small_16x64x64")
    f, _ = inputs.workload_video(wl.name)
    x, tr, st, _ = gpu_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p)
    ref = oracle_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32
    assert abs(np.linalg.norm(x) - 1) < 1e-6
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    np.testing.assert_allclose(tr["norms"], ref["norms"], rtol=1e-6)
    np.testing.assert_allclose(tr["residual"], ref["residual"], rtol=1e-3,
                               atol=1e-5 * ref["rayleigh"][-1])
    assert np.all(x >= -1e-7)       # Perron-Frobenius: from x0 >= 0 the iterate stays >= 0


ODD = [  # (shape, radii, sigmas): ragged tiles, shapes smaller than the kernel, 1-frame
    ((1, 1, 1), (2, 5, 5), (1.5, 3.0, 3.0)),
    ((1, 5, 7), (0, 2, 3), (1.0, 1.0, 2.0)),
    ((3, 17, 33), (1, 5, 5), (1.5, 3.0, 3.0)),
    ((5, 40, 70), (2, 4, 4), (1.5, 2.5, 2.5)),
    ((2, 3, 100), (3, 1, 7), (2.0, 0.8, 4.0)),
    ((9, 1, 50), (4, 0, 2), (1.2, 1.0, 1.1)),
    ((4, 33, 65), (2, 16, 16), (1.5, 6.0, 6.0)),
    ((20, 18, 9), (8, 3, 1), (3.0, 2.0, 1.0)),
]


@pytest.mark.parametrize("shape,radii,sig", ODD)
def test_odd_shapes_match_oracle(cuda_device, shape, radii, sig):
    rng = np.random.default_rng(sum(shape) + 7 * sum(radii))
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32) + 0.1
    x, tr, st, _ = gpu_power(f, x0, 4, radii, sig, 0.8, 0.3)
    ref = oracle_power(f, x0, 4, radii, sig, 0.8, 0.3)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)


def test_apply_matches_oracle(cuda_device):
    """One unnormalised y = M x with signed x and an unrelated s."""
    rng = np.random.default_rng(3)
    shape, radii, sig = (7, 45, 77), (2, 5, 5), (1.5, 3.0, 3.0)
    s = rng.random(shape, dtype=np.float32)
    f = rng.random(shape, dtype=np.float32)
    xv = rng.standard_normal(shape).astype(np.float32)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=0.6, p=0.5)
    eng.load_features(to_dev(s), to_dev(f))
    y = eng.apply(to_dev(xv)).cpu().numpy()
    eng.close()
    ref = oracle.apply_M(oracle.unary(s, 0.5), f, xv, radii, sig, 0.6)
    assert rel_l2(y, ref) < 1e-6


def test_symmetry_on_gpu(cuda_device):
    """<u, M v> = <M u, v>: the kernel applies a symmetric operator."""
    rng = np.random.default_rng(4)
    shape, radii, sig = (6, 30, 50), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    u = rng.standard_normal(shape).astype(np.float32)
    v = rng.standard_normal(shape).astype(np.float32)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    eng.load_features(to_dev(f), to_dev(f))
    Mu = eng.apply(to_dev(u)).cpu().numpy().astype(np.float64)
    Mv = eng.apply(to_dev(v)).cpu().numpy().astype(np.float64)
    eng.close()
    a, b = np.vdot(u, Mv), np.vdot(Mu, v)
    assert abs(a - b) <= 1e-5 * np.linalg.norm(u) * np.linalg.norm(Mv)


def test_rayleigh_matches_oracle(cuda_device):
    rng = np.random.default_rng(5)
    shape, radii, sig = (5, 20, 30), (1, 3, 3), (1.0, 2.0, 2.0)
    f = rng.random(shape, dtype=np.float32)
    x = rng.random(shape, dtype=np.float32)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    eng.load_features(to_dev(f), to_dev(f))
    lam, res = eng.rayleigh(to_dev(x))
    eng.close()
    ref = oracle.power_iterate(oracle.unary(f, 0.1), f, x, 1, radii, sig, 1.0)
    assert abs(lam - ref["rayleigh"][0]) < 1e-6 * abs(ref["rayleigh"][0])
    assert abs(res - ref["residual"][0]) < 1e-4 * ref["residual"][0]


def test_graph_replay_equals_eager_and_is_deterministic(cuda_device):
    wl, radii, sig = _wl("small_16x64x64")
    f, _ = inputs.workload_video(wl.name)
    a, ta, _, _ = gpu_power(f, f, 12, radii, sig, 1.0, 0.1)
    b, tb, _, _ = gpu_power(f, f, 12, radii, sig, 1.0, 0.1, flags=sf.SFSEG_NO_GRAPH)
    c, _, _, _ = gpu_power(f, f, 12, radii, sig, 1.0, 0.1)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.array_equal(ta["rayleigh"], tb["rayleigh"])


def test_repeated_calls_on_one_context(cuda_device):
    """A context replays its cached graph; a second call gives the same bits."""
    import torch
    rng = np.random.default_rng(6)
    shape = (6, 33, 47)
    f = rng.random(shape, dtype=np.float32)
    eng = sf.SFSeg(shape, radii=(2, 3, 3), sigmas=(1.5, 2, 2), alpha=1.0, p=0.1)
    d = to_dev(f)
    x1 = eng.power_iterate(d, d, d, 7).clone()
    x2 = eng.power_iterate(None, None, d, 7).clone()
    torch.cuda.synchronize()
    eng.close()
    assert torch.equal(x1, x2)


def test_zero_start_and_nonfinite_inputs(cuda_device):
    shape = (3, 10, 12)
    f = np.random.default_rng(7).random(shape, dtype=np.float32)
    x, _, st, _ = gpu_power(f, np.zeros(shape, np.float32), 3, (1, 2, 2), (1, 1, 1), 1.0, 0.1)
    assert st == sf.SFSEG_EZERONORM
    bad = f.copy()
    bad[1, 2, 3] = np.nan
    _, _, st, _ = gpu_power(bad, f, 3, (1, 2, 2), (1, 1, 1), 1.0, 0.1)
    assert st == sf.SFSEG_ENONFINITE


def test_zero_norm_step_keeps_last_iterate(cuda_device):
    """x0 supported where sp = 0 only: ||M x0|| = 0 at step 0, so the output
    stays the normalised x0 and the status is EZERONORM."""
    shape = (2, 8, 8)
    s = np.ones(shape, np.float32)
    s[0, 0, 0] = 0.0
    x0 = np.zeros(shape, np.float32)
    x0[0, 0, 0] = 3.0
    x, _, st, done = gpu_power(np.zeros(shape, np.float32), x0, 5, (1, 1, 1), (1, 1, 1), 1.0,
                               1.0, s=s, tol=1e-9)
    assert st == sf.SFSEG_EZERONORM and done == 0
    assert x[0, 0, 0] == 1.0 and np.count_nonzero(x) == 1


def test_early_stop_on_residual(cuda_device):
    rng = np.random.default_rng(8)
    shape, radii, sig = (4, 8, 8), (1, 2, 2), (1.0, 1.5, 1.5)
    f = rng.random(shape, dtype=np.float32)
    x, tr, st, done = gpu_power(f, f, 3000, radii, sig, 1.0, 0.1, tol=1e-4)
    assert st == sf.SFSEG_OK and 0 < done < 3000
    assert tr["residual"][-1] < 1e-4 * tr["rayleigh"][-1]
    assert tr["residual"][-2] >= 1e-4 * tr["rayleigh"][-2]
    ref = oracle.power_iterate(oracle.unary(f, 0.1), f, f, done, radii, sig, 1.0)
    assert rel_l2(x, ref["x"]) < TOL_F32


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_low_precision_storage_small(cuda_device, storage):
    """BF16/FP16 storage, FP32 arithmetic: the final iterate is within 1e-3
    rel-L2 of the FP64 oracle fed the same rounded sp, f, x0."""
    wl, radii, sig = _wl("small_16x64x64")
    f, _ = inputs.workload_video(wl.name)
    sp = (f.astype(np.float32) ** np.float32(wl.p)).astype(np.float32)
    x, tr, st, _ = gpu_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p, s=sp, storage=storage,
                             flags=sf.SFSEG_S_IS_SP)
    ref = oracle.power_iterate(oracle.to_storage(sp, storage), oracle.to_storage(f, storage),
                               oracle.to_storage(f, storage), wl.iters, radii, sig, wl.alpha)
    assert st == sf.SFSEG_OK
    err = rel_l2(x, ref["x"])
    assert err < TOL_LOWP, err
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-3)


def test_batched_equals_single_runs(cuda_device):
    """Uneven videos in one launch per step: each equals its own run."""
    import torch
    shapes = [(5, 24, 40), (9, 31, 17), (3, 40, 64), (1, 7, 9)]
    rng = np.random.default_rng(9)
    fs = [rng.random(s, dtype=np.float32) for s in shapes]
    radii, sig = (2, 4, 4), (1.5, 2.5, 2.5)
    eng = sf.SFSeg(batch_shapes=shapes, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    xs = [to_dev(f) for f in fs]
    eng.power_iterate_batched([to_dev(f) for f in fs], [to_dev(f) for f in fs], xs, 6)
    torch.cuda.synchronize()
    traces = [eng.trace(v) for v in range(len(shapes))]
    eng.close()
    for f, xb, tb in zip(fs, xs, traces):
        # each voxel's arithmetic is the same; only the FP64 norm sums are
        # grouped differently when the batch is split across CTAs
        xs1, ts1, _, _ = gpu_power(f, f, 6, radii, sig, 1.0, 0.1)
        assert rel_l2(xb.cpu().numpy(), xs1) < 1e-6
        np.testing.assert_allclose(tb["rayleigh"], ts1["rayleigh"], rtol=1e-6)
        ref = oracle_power(f, f, 6, radii, sig, 1.0, 0.1)
        assert rel_l2(xb.cpu().numpy(), ref["x"]) < TOL_F32


FAST = [  # radii with a specialised kernel; shapes with many CTA segment cuts
    ((40, 64, 256), (2, 5, 5), (1.5, 3.0, 3.0)),
    ((11, 37, 300), (2, 4, 4), (1.5, 2.5, 2.5)),
    ((3, 200, 130), (2, 5, 5), (1.0, 2.0, 3.0)),
]


@pytest.mark.parametrize("shape,radii,sig", FAST)
def test_specialised_kernel_matches_oracle_and_generic(cuda_device, shape, radii, sig):
    rng = np.random.default_rng(sum(shape))
    f = rng.random(shape, dtype=np.float32)
    x, tr, st, _ = gpu_power(f, f, 5, radii, sig, 1.0, 0.1)
    xg, trg, _, _ = gpu_power(f, f, 5, radii, sig, 1.0, 0.1, flags=sf.SFSEG_GENERIC)
    x2, _, _, _ = gpu_power(f, f, 5, radii, sig, 1.0, 0.1)
    ref = oracle_power(f, f, 5, radii, sig, 1.0, 0.1)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32
    assert rel_l2(x, xg) < 1e-6
    assert np.array_equal(x, x2)                       # deterministic
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    np.testing.assert_allclose(tr["residual"], ref["residual"], rtol=1e-4)


def test_batched_bf16_equals_single_runs_and_oracle(cuda_device):
    """BF16 storage in the batched launch (the batched form runs FP32 and
    BF16): each video equals its own single-video BF16 run, and its x^K is
    within the low-precision bar of the oracle fed the same rounded operands."""
    import torch
    shapes = [(6, 30, 70), (4, 48, 33), (8, 20, 128)]
    rng = np.random.default_rng(21)
    fs = [rng.random(s, dtype=np.float32) for s in shapes]
    radii, sig = (2, 4, 4), (1.5, 2.5, 2.5)
    eng = sf.SFSeg(batch_shapes=shapes, radii=radii, sigmas=sig, alpha=1.0, p=0.1, storage="bf16")
    xs = [to_dev(f) for f in fs]
    eng.power_iterate_batched([to_dev(f) for f in fs], [to_dev(f) for f in fs], xs, 5)
    torch.cuda.synchronize()
    eng.close()
    for f, xb in zip(fs, xs):
        x1, _, st, _ = gpu_power(f, f, 5, radii, sig, 1.0, 0.1, storage="bf16")
        assert st == sf.SFSEG_OK
        assert rel_l2(xb.cpu().numpy(), x1) < 1e-5
        ref = oracle_power(f, f, 5, radii, sig, 1.0, 0.1, storage="bf16")
        assert rel_l2(xb.cpu().numpy(), ref["x"]) < TOL_LOWP


def test_batched_many_small_videos(cuda_device):
    """More videos than CTAs (one voxel, single rows and columns, a video
    wider than one tile), in one launch per step: each equals its own run."""
    import torch
    rng = np.random.default_rng(5)
    shapes = [(1, 1, 1), (1, 1, 9), (3, 1, 5), (2, 7, 1)]
    shapes += [tuple(int(v) for v in rng.integers(1, 12, size=3)) for _ in range(200)]
    shapes += [(12, 40, 300)]
    fs = [0.9 * rng.random(s, dtype=np.float32) + 0.05 for s in shapes]
    radii, sig = (2, 5, 5), (1.5, 3.0, 3.0)
    eng = sf.SFSeg(batch_shapes=shapes, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    xs = [to_dev(f) for f in fs]
    eng.power_iterate_batched([to_dev(f) for f in fs], [to_dev(f) for f in fs], xs, 4)
    torch.cuda.synchronize()
    eng.close()
    for k in list(range(8)) + [len(shapes) - 1]:
        x1, _, _, _ = gpu_power(fs[k], fs[k], 4, radii, sig, 1.0, 0.1)
        assert rel_l2(xs[k].cpu().numpy(), x1) < 1e-6, (k, shapes[k])
    one = xs[0].cpu().numpy()
    assert one.shape == (1, 1, 1) and abs(float(one.ravel()[0]) - 1.0) < 1e-6   # x = 1 for one voxel
    for k in range(len(shapes)):
        x = xs[k].cpu().numpy().astype(np.float64)
        assert abs(np.linalg.norm(x) - 1.0) < 1e-5 and x.min() >= -1e-7, (k, shapes[k])
