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

from _helpers import TOL_F32, rel_l2

pytestmark = pytest.mark.gpu


def _params(shape, radii=(2, 5, 5), sig=(1.5, 3.0, 3.0)):
    p = sf.sfseg_default_params(*shape)
    p.rt, p.ry, p.rx = radii
    p.sigma_t, p.sigma_y, p.sigma_x = sig
    p.alpha, p.p = 1.0, 0.1
    return p


def test_noalloc_matches_power_iterate_twice(cuda_device):
    """Two calls in a row (different volumes, the second reusing the array
    the first left behind) each match sfseg_power_iterate."""
    import torch
    shape, K = (7, 45, 90), 12
    rng = np.random.default_rng(31)
    for call in range(2):
        f = rng.random(shape, dtype=np.float32)
        x0 = (rng.random(shape, dtype=np.float32) + 0.1) if call else f.copy()
        d_f = torch.from_numpy(f).cuda()
        x_na = torch.from_numpy(x0).cuda()
        trace = torch.zeros((K, 3), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        sf.sfseg_power_iterate_noalloc(_params(shape), d_f.data_ptr(), d_f.data_ptr(),
                                       x_na.data_ptr(), K, trace.data_ptr(), stream)
        eng = sf.SFSeg(shape, radii=(2, 5, 5), sigmas=(1.5, 3.0, 3.0), alpha=1.0, p=0.1,
                       flags=sf.SFSEG_GENERIC)
        x_ref = eng.power_iterate(d_f, d_f, torch.from_numpy(x0).cuda(), K)
        torch.cuda.synchronize()
        tr_ref = eng.trace()
        eng.close()
        assert rel_l2(x_na.cpu().numpy(), x_ref.cpu().numpy()) < TOL_F32
        np.testing.assert_allclose(trace[:, 0].cpu().numpy(), tr_ref["rayleigh"], rtol=1e-6)
        np.testing.assert_allclose(trace[:, 2].cpu().numpy(), tr_ref["norms"], rtol=1e-6)


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
