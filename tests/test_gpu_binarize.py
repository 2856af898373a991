"""Binarisation schedule (Alg. 1 Step 3, Sec. 4) on the GPU against the oracle.

Each projection p = 1 / (1 + exp(-beta (u - tau))) multiplies a perturbation
of u by at most the logistic slope beta / 4, so after n projections the FP32
bar of the plain iteration (1e-5 rel-L2) becomes 1e-5 * max(1, beta / 4)^n.
The mask is compared exactly where the oracle's u is farther than 1e-4 from
theta; closer voxels may flip with the FP32 rounding of x.
"""
import numpy as np
import pytest

import oracle
from oracle import binarize
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs
from _helpers import TOL_F32, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _run(f, K, radii, sig, k0, beta, tau, theta, p=0.1, x0=None, storage="f32"):
    import torch
    eng = sf.SFSeg(f.shape, radii=radii, sigmas=sig, alpha=1.0, p=p, storage=storage)
    try:
        x = to_dev(f if x0 is None else x0)
        x, mask = eng.power_iterate_binarized(to_dev(f), to_dev(f), x, K, k0=k0, beta=beta, tau=tau,
                                              theta=theta, out=x)
        torch.cuda.synchronize()
        return x.cpu().numpy(), mask.cpu().numpy(), eng.trace(), eng.sync_status()
    finally:
        eng.close()


def _oracle(f, K, radii, sig, k0, beta, tau, theta, p=0.1, x0=None):
    sp = oracle.unary(np.asarray(f, np.float64), p)
    return binarize.power_iterate_binarized(sp, np.asarray(f, np.float64),
                                            np.asarray(f if x0 is None else x0, np.float64), K, radii,
                                            sig, 1.0, k0, beta, tau, theta)


def _check_mask(x, mask, ref, theta):
    # the GPU mask is the FP32 threshold of the GPU's own x
    np.testing.assert_array_equal(mask, (x >= np.float32(theta) * x.max()).astype(np.uint8))
    u = ref["x"] / ref["x"].max()
    far = np.abs(u - theta) > 1e-4
    np.testing.assert_array_equal(mask[far], ref["mask"][far])
    assert far.mean() > 0.99


@pytest.mark.parametrize("case", [
    ((16, 64, 64), (3, 3, 3), (1.5, 2.0, 2.0), 10, 5, 4.0, 0.5, 0.5),
    ((5, 40, 70), (2, 5, 5), (1.5, 3.0, 3.0), 9, 3, 4.0, 0.4, 0.3),
    ((3, 17, 33), (1, 5, 5), (1.5, 3.0, 3.0), 6, 1, 2.0, 0.6, 0.7),
])
def test_binarized_matches_oracle(cuda_device, case):
    shape, radii, sig, K, k0, beta, tau, theta = case
    f, _ = inputs.make_video(*shape, inputs.config_seed(7, K), 1)
    x, mask, tr, st = _run(f, K, radii, sig, k0, beta, tau, theta)
    ref = _oracle(f, K, radii, sig, k0, beta, tau, theta)
    n_proj = max(0, K - k0)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32 * max(1.0, beta / 4) ** n_proj
    assert abs(np.linalg.norm(x.astype(np.float64)) - 1) < 1e-6
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-5)
    _check_mask(x, mask, ref, theta)


def test_binarized_default_schedule(cuda_device):
    """k0 = 3, beta = 10, tau = theta = 1/2 on the 16 x 64 x 64 video, 10 steps."""
    wl = inputs.WORKLOADS["small_16x64x64"]
    f, truth = inputs.workload_video(wl.name)
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    K, k0, beta = 10, 3, 10.0
    x, mask, _, st = _run(f, K, radii, sig, k0, beta, 0.5, 0.5)
    ref = _oracle(f, K, radii, sig, k0, beta, 0.5, 0.5)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_F32 * (beta / 4) ** (K - k0)
    _check_mask(x, mask, ref, 0.5)
    # the binarised iterate is closer to a 0/1 vector than the plain one
    # (Sec. 4): fewer voxels with u = x / max(x) strictly between 0.1 and 0.9
    plain = oracle.power_iterate(oracle.unary(f.astype(np.float64), 0.1), f.astype(np.float64),
                                 f.astype(np.float64), K, radii, sig, 1.0)["x"]
    mid = lambda v: float(np.mean((v / v.max() > 0.1) & (v / v.max() < 0.9)))
    assert abs(mid(x) - mid(ref["x"])) < 1e-3
    assert mid(x) < 0.5 * mid(plain)


def test_binarized_without_projection_equals_plain(cuda_device):
    """k0 >= K: the same x^K as sfseg_power_iterate."""
    import torch
    f, _ = inputs.make_video(6, 40, 72, 99, 1)
    radii, sig = (2, 5, 5), (1.5, 3.0, 3.0)
    x, _, _, _ = _run(f, 8, radii, sig, 8, 10.0, 0.5, 0.5)
    eng = sf.SFSeg(f.shape, radii=radii, sigmas=sig, alpha=1.0, p=0.1)
    xp = eng.power_iterate(to_dev(f), to_dev(f), to_dev(f), 8)
    torch.cuda.synchronize()
    eng.close()
    assert rel_l2(x, xp.cpu().numpy()) < 1e-6


def test_binarized_bad_schedule(cuda_device):
    f = np.ones((2, 8, 8), np.float32)
    eng = sf.SFSeg(f.shape, radii=(1, 1, 1), sigmas=(1.0, 1.0, 1.0))
    try:
        for kw in ({"k0": 0}, {"beta": -1.0}, {"tau": float("nan")}):
            with pytest.raises(sf.SFSegError) as ei:
                eng.power_iterate_binarized(to_dev(f), to_dev(f), to_dev(f), 4, **kw)
            assert ei.value.status == sf.SFSEG_EINVAL
    finally:
        eng.close()
