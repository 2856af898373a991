"""The cluster path (all K power steps of one small video in one thread-block
cluster, the video resident in shared memory) against the FP64 oracle, and
its place among the other step paths."""
import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs

from _helpers import TOL_F32, TOL_LOWP, gpu_power, oracle_power, rel_l2, to_dev

pytestmark = pytest.mark.gpu

CL = sf.SFSEG_CLUSTER


def _engine(shape, radii, sig, flags=CL, **kw):
    return sf.SFSeg(shape, radii=radii, sigmas=sig, flags=flags, **kw)


def test_cluster_small_workload_matches_oracle(cuda_device):
    """16x64x64, 7x7x7 Gaussian, 30 steps from x0 = f: 16 CTAs of 16x16 tiles."""
    wl = inputs.WORKLOADS["small_16x64x64"]
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    f, _ = inputs.workload_video(wl.name)
    eng = _engine(f.shape, radii, sig, alpha=wl.alpha, p=wl.p)
    info = eng.path()
    eng.close()
    assert info["path"] == "cluster" and info["fused_ctas"] == 16
    x, tr, st, n = gpu_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p, flags=CL)
    ref = oracle_power(f, f, wl.iters, radii, sig, wl.alpha, wl.p)
    assert st == sf.SFSEG_OK and n == wl.iters
    assert rel_l2(x, ref["x"]) < TOL_F32
    assert abs(np.linalg.norm(x) - 1) < 1e-6
    np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
    np.testing.assert_allclose(tr["norms"], ref["norms"], rtol=1e-6)
    np.testing.assert_allclose(tr["residual"], ref["residual"], rtol=1e-3,
                               atol=1e-5 * ref["rayleigh"][-1])
    assert np.all(x >= -1e-7)


SHAPES = [  # ragged 16-column tiles and 8-row chunks, one CTA, one frame, 16 CTAs in a row
    ((1, 1, 1), (2, 5, 5), (1.5, 3.0, 3.0)),
    ((12, 8, 16), (2, 5, 5), (1.5, 3.0, 3.0)),
    ((3, 17, 33), (2, 4, 4), (1.5, 2.5, 2.5)),
    ((5, 40, 70), (2, 4, 4), (1.5, 2.5, 2.5)),
    ((20, 20, 20), (3, 3, 3), (1.5, 2.0, 2.0)),
    ((7, 33, 50), (2, 4, 4), (1.2, 2.0, 3.0)),
    ((2, 9, 250), (3, 3, 3), (2.0, 1.0, 2.5)),
    ((1, 64, 64), (3, 3, 3), (1.5, 2.0, 2.0)),
    ((9, 5, 3), (3, 3, 3), (1.0, 1.0, 1.0)),
]


@pytest.mark.parametrize("shape,radii,sig", SHAPES)
def test_cluster_shapes_match_oracle(cuda_device, shape, radii, sig):
    rng = np.random.default_rng(sum(shape) + 11 * sum(radii))
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32) + 0.1
    for K in (4, 5):   # the result leaves the cluster from either tile buffer
        x, tr, st, _ = gpu_power(f, x0, K, radii, sig, 0.8, 0.3, flags=CL)
        ref = oracle_power(f, x0, K, radii, sig, 0.8, 0.3)
        assert st == sf.SFSEG_OK
        assert rel_l2(x, ref["x"]) < TOL_F32
        np.testing.assert_allclose(tr["rayleigh"], ref["rayleigh"], rtol=1e-6)
        np.testing.assert_allclose(tr["norms"], ref["norms"], rtol=1e-6)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_cluster_low_precision_storage(cuda_device, storage):
    rng = np.random.default_rng(23)
    shape, radii, sig = (6, 40, 52), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    x, _, st, _ = gpu_power(f, f, 12, radii, sig, 1.0, 0.1, storage=storage, flags=CL)
    ref = oracle_power(f, f, 12, radii, sig, 1.0, 0.1, storage=storage)
    assert st == sf.SFSEG_OK
    assert rel_l2(x, ref["x"]) < TOL_LOWP


def test_cluster_early_stop_and_zero_norm(cuda_device):
    """tol > 0: the iterate of the converged step leaves through the ping-pong
    buffer finish reads; ||M x0|| = 0 stops at step 0 with x0 returned."""
    rng = np.random.default_rng(9)
    shape, radii, sig = (4, 8, 8), (3, 3, 3), (1.0, 1.5, 1.5)
    f = rng.random(shape, dtype=np.float32)
    x, tr, st, done = gpu_power(f, f, 3000, radii, sig, 1.0, 0.1, tol=1e-4, flags=CL)
    assert st == sf.SFSEG_OK and 0 < done < 3000
    assert tr["residual"][-1] < 1e-4 * tr["rayleigh"][-1]
    assert tr["residual"][-2] >= 1e-4 * tr["rayleigh"][-2]
    ref = oracle.power_iterate(oracle.unary(f, 0.1), f, f, done, radii, sig, 1.0)
    assert rel_l2(x, ref["x"]) < TOL_F32
    s = np.ones((2, 8, 8), np.float32)
    s[0, 0, 0] = 0.0
    x0 = np.zeros((2, 8, 8), np.float32)
    x0[0, 0, 0] = 3.0
    x, _, st, done = gpu_power(np.zeros((2, 8, 8), np.float32), x0, 5, (2, 4, 4), (1, 1, 1), 1.0,
                               1.0, s=s, tol=1e-9, flags=CL)
    assert st == sf.SFSEG_EZERONORM and done == 0
    assert x[0, 0, 0] == 1.0 and np.count_nonzero(x) == 1


def test_cluster_equals_other_paths_and_is_deterministic(cuda_device):
    import torch
    wl = inputs.WORKLOADS["small_16x64x64"]
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    f_np, _ = inputs.workload_video(wl.name)
    f = to_dev(f_np)
    out = {}
    for name, flags in (("cluster", CL), ("fused", sf.SFSEG_FUSED), ("generic", 0)):
        eng = _engine(f_np.shape, radii, sig, flags=flags, alpha=wl.alpha, p=wl.p)
        xs = []
        for _ in range(2):
            x = f.clone()
            eng.power_iterate(f, f, x, 9, out=x)
            xs.append(x)
        torch.cuda.synchronize()
        tr = eng.trace()
        eng.close()
        if name == "cluster":
            assert torch.equal(xs[0], xs[1])   # fixed summation order
        out[name] = (xs[0].cpu().numpy(), tr)
    for name in ("fused", "generic"):
        assert rel_l2(out["cluster"][0], out[name][0]) < 1e-6
        np.testing.assert_allclose(out["cluster"][1]["rayleigh"], out[name][1]["rayleigh"], rtol=1e-6)


def test_autotuner_times_the_cluster_path(cuda_device):
    import torch
    wl = inputs.WORKLOADS["small_16x64x64"]
    radii, sig = (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    f_np, _ = inputs.workload_video(wl.name)
    f = to_dev(f_np)
    eng = _engine(f_np.shape, radii, sig, flags=sf.SFSEG_AUTOTUNE, alpha=wl.alpha, p=wl.p)
    try:
        x = f.clone()
        eng.power_iterate(f, f, x, wl.iters, out=x)
        torch.cuda.synchronize()
        info = eng.path()
    finally:
        eng.close()
    assert "cluster" in info["tuned_us"] and info["tuned_us"]["cluster"] > 0
    best = min(info["tuned_us"], key=info["tuned_us"].get)
    assert info["path"] == best
    ref = oracle_power(f_np, f_np, wl.iters, radii, sig, wl.alpha, wl.p)
    assert rel_l2(x.cpu().numpy(), ref["x"]) < TOL_F32


def test_cluster_context_serves_the_per_step_calls(cuda_device):
    """Rayleigh quotient and one application of M run the per-step kernels."""
    rng = np.random.default_rng(31)
    shape, radii, sig = (8, 24, 40), (2, 5, 5), (1.5, 3.0, 3.0)
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32)
    eng = _engine(shape, radii, sig, alpha=0.7, p=0.2)
    try:
        assert eng.path()["path"] == "cluster"
        fd = to_dev(f)
        eng.load_features(fd, fd)
        r, _ = eng.rayleigh(to_dev(x0))
        y = eng.apply(to_dev(x0)).cpu().numpy()
        with pytest.raises(sf.SFSegError) as ei:
            eng.debug_inject_timeout(1)
        assert ei.value.status == sf.SFSEG_EUNSUPPORTED
    finally:
        eng.close()
    sp = oracle.unary(f.astype(np.float64), 0.2)
    My = oracle.apply_M(sp, f.astype(np.float64), x0.astype(np.float64), radii, sig, 0.7)
    assert rel_l2(y, My) < TOL_F32
    assert abs(r - float(np.dot(x0.ravel(), My.ravel()) / np.dot(x0.ravel(), x0.ravel()))) < 1e-5 * abs(r)


def test_cluster_rejects_videos_it_cannot_hold(cuda_device):
    for shape, radii in (((16, 64, 64), (1, 1, 1)),       # radii not compiled for the cluster
                         ((16, 64, 64), (2, 5, 5)),       # frames do not fit a CTA's shared memory
                         ((4, 16, 300), (3, 3, 3)),       # more than 16 tiles
                         ((10, 60, 107), (2, 5, 5))):
        with pytest.raises(sf.SFSegError) as ei:
            _engine(shape, radii, (1.5, 2.0, 2.0))
        assert ei.value.status == sf.SFSEG_EUNSUPPORTED
