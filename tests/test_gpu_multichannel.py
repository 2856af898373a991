"""Multi-channel pairwise features (Eq. 9) on the GPU against the FP64 oracle.

M_ij = sp_i sp_j sum_c [1 - alpha (f_ci - f_cj)^2] G_ij, evaluated by the
any-radius step kernel with C + 2 convolutions; the oracle sums the same
per-channel Taylor affinities edge by edge.
"""
import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs
from _helpers import TOL_F32, TOL_LOWP, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _features(shape, C, seed):
    """s from a seeded video, channel 0 = s, further channels seeded videos of
    their own (stand-ins for the paper's two optical-flow magnitudes)."""
    nf, h, w = shape
    s, _ = inputs.make_video(nf, h, w, seed, 1)
    chans = [s] + [inputs.make_video(nf, h, w, seed + 100 * c, 1)[0] for c in range(1, C)]
    return s, np.ascontiguousarray(np.stack(chans).astype(np.float32))


def _gpu(shape, s, f, x0, K, radii, sig, alpha, p, storage="f32", nchan=1):
    import torch
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=alpha, p=p, storage=storage, nchan=nchan)
    try:
        x = to_dev(x0)
        eng.power_iterate(to_dev(s), to_dev(f), x, K, out=x)
        torch.cuda.synchronize()
        return x.cpu().numpy(), eng.trace(), eng.sync_status()
    finally:
        eng.close()


CASES = [  # (shape, C, radii, sigmas, K)
    ((8, 40, 70), 2, (2, 5, 5), (1.5, 3.0, 3.0), 20),
    ((5, 33, 47), 3, (1, 3, 3), (1.0, 2.0, 2.0), 15),
    ((6, 20, 30), 4, (2, 4, 4), (1.5, 2.5, 2.5), 12),
    ((1, 1, 1), 2, (2, 5, 5), (1.5, 3.0, 3.0), 3),
    ((3, 17, 100), 2, (1, 16, 2), (1.0, 6.0, 1.0), 8),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_multichannel_power_matches_oracle(cuda_device, case):
    shape, C, radii, sig, K = CASES[case]
    s, f = _features(shape, C, 1907 + case)
    x, tr, st = _gpu(shape, s, f, s, K, radii, sig, 1.0, 0.1, nchan=C)
    ref = oracle.power_iterate(oracle.unary(s, 0.1), f.astype(np.float64), s, K, radii, sig, 1.0)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    assert np.all(x >= -1e-7)


def test_multichannel_apply_matches_oracle(cuda_device):
    """One unnormalised y = M x, signed x, C = 2, alpha and p away from 1."""
    rng = np.random.default_rng(5)
    shape, radii, sig = (6, 37, 61), (2, 5, 5), (1.5, 3.0, 3.0)
    s = rng.random(shape, dtype=np.float32)
    f = rng.random((2,) + shape, dtype=np.float32)
    xv = rng.standard_normal(shape).astype(np.float32)
    eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=0.6, p=0.5, nchan=2)
    eng.load_features(to_dev(s), to_dev(f))
    y = eng.apply(to_dev(xv)).cpu().numpy()
    eng.close()
    ref = oracle.apply_M(oracle.unary(s, 0.5), f.astype(np.float64), xv, radii, sig, 0.6)
    assert rel_l2(y, ref) < 1e-6
    # sampled outputs one by one from the oracle's per-voxel routine
    idx = rng.integers(0, int(np.prod(shape)), 40)
    ref_at = oracle.apply_M_at(oracle.unary(s, 0.5), f.astype(np.float64), xv, radii, sig, 0.6, idx)
    got = y.ravel()[idx]
    np.testing.assert_allclose(got, ref_at, rtol=2e-5, atol=2e-5 * np.abs(ref).max())


def test_identical_channels_match_single_channel(cuda_device):
    """C copies of one channel: C M, so the same iterates and C times the
    Rayleigh quotient of the single-channel (specialised-kernel) run."""
    shape, radii, sig, K = (10, 48, 120), (2, 5, 5), (1.5, 3.0, 3.0), 25
    s, _ = _features(shape, 1, 77)
    f2 = np.ascontiguousarray(np.stack([s, s]))
    x1, tr1, _ = _gpu(shape, s, s, s, K, radii, sig, 1.0, 0.1)
    x2, tr2, _ = _gpu(shape, s, f2, s, K, radii, sig, 1.0, 0.1, nchan=2)
    assert rel_l2(x2, x1) < 1e-6
    np.testing.assert_allclose(tr2["rayleigh"], 2 * np.asarray(tr1["rayleigh"]), rtol=1e-6)


def test_multichannel_bf16_storage(cuda_device):
    """BF16 storage, C = 2: against the oracle on the same rounded operands."""
    shape, radii, sig, K = (6, 40, 72), (2, 5, 5), (1.5, 3.0, 3.0), 15
    s, f = _features(shape, 2, 31)
    x, _, st = _gpu(shape, s, f, s, K, radii, sig, 1.0, 0.1, storage="bf16", nchan=2)
    sp = oracle.to_storage(s.astype(np.float32) ** np.float32(0.1), "bf16")
    ref = oracle.power_iterate(sp, oracle.to_storage(f, "bf16"), oracle.to_storage(s, "bf16"), K,
                               radii, sig, 1.0)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_LOWP


def test_multichannel_batched_matches_single(cuda_device):
    """Three videos of different shapes, C = 2, one launch per step: each
    equals its own single-video run."""
    import torch
    dims = [(4, 30, 50), (6, 21, 33), (3, 40, 64)]
    radii, sig, K = (1, 4, 4), (1.5, 2.5, 2.5), 10
    feats = [_features(d, 2, 500 + i) for i, d in enumerate(dims)]
    eng = sf.SFSeg(batch_shapes=dims, radii=radii, sigmas=sig, alpha=1.0, p=0.1, nchan=2)
    ss = [to_dev(s) for s, _ in feats]
    fs = [to_dev(f) for _, f in feats]
    xs = [to_dev(s) for s, _ in feats]
    eng.power_iterate_batched(ss, fs, xs, K)
    torch.cuda.synchronize()
    eng.close()
    for (s, f), d, xb in zip(feats, dims, xs):
        x1, _, _ = _gpu(d, s, f, s, K, radii, sig, 1.0, 0.1, nchan=2)
        assert rel_l2(xb.cpu().numpy(), x1) < 1e-6


@pytest.mark.parametrize("C,radii,sig", [(2, (2, 5, 5), (1.5, 3.0, 3.0)), (3, (2, 4, 4), (1.5, 2.5, 2.5))])
def test_channel_passes_match_any_radius_kernel(cuda_device, C, radii, sig):
    """FP32 storage runs several channels as one specialised pass per channel
    (Eq. 9 as a sum); it must agree with the any-radius kernel's C + 2
    convolutions: iterates, Rayleigh trace, y = Mx and sfseg_rayleigh."""
    import torch
    shape, K = (9, 50, 130), 12
    s, f = _features(shape, C, 4242 + C)
    outs = []
    for flags in (0, sf.SFSEG_GENERIC):
        eng = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=0.9, p=0.1, nchan=C, flags=flags)
        try:
            x = eng.power_iterate(to_dev(s), to_dev(f), to_dev(s), K)
            torch.cuda.synchronize()
            tr = eng.trace()
            y = eng.apply(to_dev(s))
            lam, res = eng.rayleigh(to_dev(s))
            outs.append((x.cpu().numpy(), tr, y.cpu().numpy(), lam, res))
        finally:
            eng.close()
    (x1, t1, y1, l1, r1), (x2, t2, y2, l2, r2) = outs
    assert rel_l2(x1, x2) < 1e-6
    np.testing.assert_allclose(t1["rayleigh"], t2["rayleigh"], rtol=1e-6)
    assert rel_l2(y1, y2) < 1e-6
    assert abs(l1 - l2) < 1e-6 * abs(l2)


def test_channel_passes_batched_match_single(cuda_device):
    """The per-channel passes of the specialised kernel in a batched context
    (per-video partial sums): each video equals its own single-video run and
    the any-radius kernel's result."""
    import torch
    dims = [(5, 30, 120), (7, 26, 90), (4, 40, 112)]
    radii, sig, K = (2, 4, 4), (1.5, 2.5, 2.5), 9
    feats = [_features(d, 2, 700 + i) for i, d in enumerate(dims)]
    res = {}
    for flags in (0, sf.SFSEG_GENERIC):
        eng = sf.SFSeg(batch_shapes=dims, radii=radii, sigmas=sig, alpha=1.0, p=0.1, nchan=2, flags=flags)
        xs = [to_dev(s) for s, _ in feats]
        eng.power_iterate_batched([to_dev(s) for s, _ in feats], [to_dev(f) for _, f in feats], xs, K)
        torch.cuda.synchronize()
        eng.close()
        res[flags] = [x.cpu().numpy() for x in xs]
    for i, ((s, f), d) in enumerate(zip(feats, dims)):
        x1, _, _ = _gpu(d, s, f, s, K, radii, sig, 1.0, 0.1, nchan=2)
        assert rel_l2(res[0][i], x1) < 1e-6
        assert rel_l2(res[0][i], res[sf.SFSEG_GENERIC][i]) < 1e-6
