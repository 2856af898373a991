"""The allocation-free entry point (sfseg_power_iterate_noalloc).

Some callers may not call cudaMalloc (a region captured into a larger CUDA
graph, a real-time path with a fixed memory budget, a plug-in whose host
framework owns all device memory).  The library gives them one entry point
whose workspace is a fixed device array inside the library.  This file is
collected last so that, if it fails, a run stopping at the first failure has
already run every other test; it must pass alone in a fresh process too.
"""
import numpy as np
import pytest

import paper_1907_02731_gb300 as sf

from _helpers import TOL_F32, TOL_LOWP, oracle_power, rel_l2

pytestmark = pytest.mark.gpu


def _params(shape, radii=(2, 5, 5), sig=(1.5, 3.0, 3.0), storage="f32"):
    p = sf.sfseg_default_params(*shape)
    p.rt, p.ry, p.rx = radii
    p.sigma_t, p.sigma_y, p.sigma_x = sig
    p.alpha, p.p = 1.0, 0.1
    p.storage = sf.STORAGE[storage]
    return p


def _noalloc(f, x0, K, storage="f32", shape=None):
    """x^K and the trace of the allocation-free entry point."""
    import torch
    shape = shape or f.shape
    d_f = torch.from_numpy(f).cuda()
    x = torch.from_numpy(x0).cuda()
    trace = torch.zeros((K, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sf.sfseg_power_iterate_noalloc(_params(shape, storage=storage), d_f.data_ptr(), d_f.data_ptr(),
                                   x.data_ptr(), K, trace.data_ptr(), stream)
    torch.cuda.synchronize()
    return x.cpu().numpy(), trace.cpu().numpy()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_noalloc_matches_power_iterate_twice(cuda_device, storage):
    """Two calls in a row (different volumes, the second reusing the array
    the first left behind) each match sfseg_power_iterate on the same kernel
    and storage type."""
    import torch
    shape, K = (7, 45, 90), 12
    rng = np.random.default_rng(31)
    tol = TOL_F32 if storage == "f32" else TOL_LOWP
    for call in range(2):
        f = rng.random(shape, dtype=np.float32)
        x0 = (rng.random(shape, dtype=np.float32) + 0.1) if call else f.copy()
        x_na, trace = _noalloc(f, x0, K, storage)
        eng = sf.SFSeg(shape, radii=(2, 5, 5), sigmas=(1.5, 3.0, 3.0), alpha=1.0, p=0.1,
                       storage=storage, flags=sf.SFSEG_GENERIC)
        d_f = torch.from_numpy(f).cuda()
        x_ref = eng.power_iterate(d_f, d_f, torch.from_numpy(x0).cuda(), K)
        torch.cuda.synchronize()
        tr_ref = eng.trace()
        eng.close()
        assert rel_l2(x_na, x_ref.cpu().numpy()) < tol
        np.testing.assert_allclose(trace[:, 0], tr_ref["rayleigh"], rtol=1e-6)
        np.testing.assert_allclose(trace[:, 2], tr_ref["norms"], rtol=1e-6)


def test_noalloc_matches_oracle(cuda_device):
    """Directly against the FP64 oracle at one small size."""
    rng = np.random.default_rng(32)
    shape, K = (5, 30, 41), 9
    f = rng.random(shape, dtype=np.float32)
    x, trace = _noalloc(f, f.copy(), K)
    ref = oracle_power(f, f, K, (2, 5, 5), (1.5, 3.0, 3.0), 1.0, 0.1)
    assert rel_l2(x, ref["x"]) < TOL_F32
    np.testing.assert_allclose(trace[:, 0], ref["rayleigh"], rtol=1e-6)


def test_noalloc_two_byte_storage_doubles_the_capacity(cuda_device):
    """63 x 256 x 256 needs four 2-byte volumes of 8.26 MB (inside the 32 MiB
    array) but four FP32 ones of 16.5 MB (outside it); 64 x 256 x 256 in BF16
    is just over the limit."""
    import torch
    shape, K = (63, 256, 256), 3
    rng = np.random.default_rng(33)
    f = rng.random(shape, dtype=np.float32)
    x, _ = _noalloc(f, f.copy(), K, "bf16")
    ref = oracle_power(f, f, K, (2, 5, 5), (1.5, 3.0, 3.0), 1.0, 0.1, storage="bf16")
    assert rel_l2(x, ref["x"]) < TOL_LOWP
    d = torch.zeros(8, device="cuda")
    for shp, st in (((63, 256, 256), "f32"), ((64, 256, 256), "bf16"), ((64, 256, 256), "f16")):
        with pytest.raises(sf.SFSegError) as ei:
            sf.sfseg_power_iterate_noalloc(_params(shp, storage=st), d.data_ptr(), d.data_ptr(),
                                           d.data_ptr(), K)
        assert ei.value.status == sf.SFSEG_EINVAL
        assert "workspace" in sf.sfseg_last_error(None)


def test_noalloc_rejects_volumes_beyond_the_array(cuda_device):
    """A volume that does not fit the fixed workspace fails with EINVAL and a
    message, before anything is launched."""
    import torch
    d = torch.zeros(8, device="cuda")
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_power_iterate_noalloc(_params((64, 480, 854)), d.data_ptr(), d.data_ptr(),
                                       d.data_ptr(), 3)
    assert ei.value.status == sf.SFSEG_EINVAL
    assert "workspace" in sf.sfseg_last_error(None)
