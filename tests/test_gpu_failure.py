"""Failure detection without a GPU fault, and writes confined to the caller's
buffers.

* A device-side wait that runs out: sfseg_debug_inject_timeout makes the first
  x-pass warp of every CTA wait on a barrier nothing arrives on; the wait gives
  up after its time limit, the other waits of the CTA give up at once, the
  step reports SFSEG_ETIMEOUT, and the same context then computes the same
  result as before, bit for bit.
* Guard bands: every buffer the library writes for the caller sits inside a
  larger allocation whose margins hold a pattern that must survive the call.
"""
import time

import numpy as np
import pytest

import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs
from paper_1907_02731_gb300.autograd import make_engine
from _helpers import to_dev

pytestmark = pytest.mark.gpu

SHAPE, RADII, SIG = (6, 40, 120), (2, 5, 5), (1.5, 3.0, 3.0)


def _video():
    f, _ = inputs.make_video(*SHAPE, inputs.config_seed(9, 1), 1)
    return to_dev(f)


def test_injected_timeout_is_reported_and_recovers(cuda_device):
    import torch
    f = _video()
    eng = sf.SFSeg(SHAPE, radii=RADII, sigmas=SIG)
    try:
        ref = eng.power_iterate(f, f, f, 6)
        assert eng.sync_status() == sf.SFSEG_OK
        eng.debug_inject_timeout(1)
        t0 = time.time()
        x = eng.power_iterate(f, f, f, 6)
        st = eng.sync_status()
        dt = time.time() - t0
        assert st == sf.SFSEG_ETIMEOUT
        assert dt < 10.0                      # one wait limit (1 s), not a hang
        assert torch.isfinite(x).all()        # the last valid iterate was returned
        again = eng.power_iterate(f, f, f, 6)
        assert eng.sync_status() == sf.SFSEG_OK
        assert torch.equal(again, ref)
    finally:
        eng.close()


def test_injection_needs_the_specialised_kernel(cuda_device):
    eng = sf.SFSeg(SHAPE, radii=RADII, sigmas=SIG, flags=sf.SFSEG_GENERIC)
    try:
        with pytest.raises(sf.SFSegError) as ei:
            eng.debug_inject_timeout(1)
        assert ei.value.status == sf.SFSEG_EUNSUPPORTED
    finally:
        eng.close()


G = 4099          # guard elements on each side; odd, so the caller's views are only 4-byte aligned


def _guarded(n, dtype, fill):
    import torch
    buf = torch.full((n + 2 * G,), fill, dtype=dtype, device="cuda")
    return buf, buf[G:G + n]


def _guards_intact(buf, n, fill):
    import torch
    lo, hi = buf[:G], buf[G + n:]
    return bool(torch.all(lo == fill)) and bool(torch.all(hi == fill))


@pytest.mark.parametrize("flags", [0, sf.SFSEG_GENERIC])
def test_writes_stay_inside_caller_buffers(cuda_device, flags):
    import torch
    f = _video()
    n = f.numel()
    eng = sf.SFSeg(SHAPE, radii=RADII, sigmas=SIG, flags=flags)
    try:
        bx, x = _guarded(n, torch.float32, 7.25)
        x.copy_(f.view(-1))
        eng.power_iterate(f, f, x.view(SHAPE), 5, out=x.view(SHAPE))
        by, y = _guarded(n, torch.float32, -3.5)
        eng.apply(f, out=y.view(SHAPE))
        torch.cuda.synchronize()
        assert _guards_intact(bx, n, 7.25) and _guards_intact(by, n, -3.5)
        assert torch.isfinite(x).all() and torch.isfinite(y).all()
    finally:
        eng.close()


def test_binarized_and_adjoint_writes_stay_inside(cuda_device):
    import torch
    f = _video()
    n = f.numel()
    eng = sf.SFSeg(SHAPE, radii=RADII, sigmas=SIG)
    try:
        bx, x = _guarded(n, torch.float32, 1.5)
        x.copy_(f.view(-1))
        xv, mask = eng.power_iterate_binarized(f, f, x.view(SHAPE), 6, out=x.view(SHAPE))
        torch.cuda.synchronize()
        assert _guards_intact(bx, n, 1.5)
        assert mask.shape == SHAPE and int(mask.max()) <= 1
    finally:
        eng.close()
    eng = make_engine(SHAPE, radii=RADII, sigmas=SIG, alpha=1.0, p=1.0, ckpt_every=4)
    try:
        eng.power_iterate(f, f, f, 9)
        g = torch.rand_like(f)
        outs = [_guarded(n, torch.float32, 2.75) for _ in range(3)]
        gsp, gf, gx0 = (o[1].view(SHAPE) for o in outs)
        sf.sfseg_adjoint(eng.ctx, g.data_ptr(), gsp.data_ptr(), gf.data_ptr(), gx0.data_ptr(),
                         sf._stream_handle())
        torch.cuda.synchronize()
        for buf, _ in outs:
            assert _guards_intact(buf, n, 2.75)
        assert all(torch.isfinite(t).all() for t in (gsp, gf, gx0))
    finally:
        eng.close()


@pytest.mark.parametrize("alpha,scale2,expect", [(1.0, 1.0, 0), (1.5, 1.0, 1), (1.0, 2.0, 1)])
def test_negative_affinity_warning(cuda_device, alpha, scale2, expect):
    """alpha * (max f - min f)^2 > 1 on some channel: the Taylor affinity can
    be negative and Perron-Frobenius no longer applies; the feature load
    reports it (the features here span [0, 1] before scaling)."""
    f = _video()
    f = (f - f.min()) / (f.max() - f.min())          # range exactly 1
    two = torch_stack([f, f * scale2])
    eng = sf.SFSeg(SHAPE, radii=RADII, sigmas=SIG, alpha=alpha, nchan=2)
    try:
        assert eng.warnings() == 0                   # nothing loaded yet
        eng.load_features(f, two)
        assert eng.warnings() == expect * sf.SFSEG_WARN_NEGATIVE_M
    finally:
        eng.close()


def torch_stack(ts):
    import torch
    return torch.stack(ts).contiguous()
