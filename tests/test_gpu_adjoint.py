"""The hand-written adjoint (sfseg_adjoint, through the C-ABI) against the
FP64 oracle's reverse mode, and its invariants."""
import numpy as np
import pytest

import oracle
import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import inputs
from paper_1907_02731_gb300.autograd import SFSegPower, make_engine

from _helpers import rel_l2, to_dev

pytestmark = pytest.mark.gpu

TOL_ADJ = 1e-4     # FP32 adjoint vs FP64 oracle adjoint, relative L2


def _gpu_grads(sp, f, x0, K, radii, sig, alpha, target, ckpt=8):
    import torch
    eng = make_engine(sp.shape, radii=radii, sigmas=sig, alpha=alpha, p=1.0, ckpt_every=ckpt)
    x = eng.power_iterate(to_dev(sp), to_dev(f), to_dev(x0), K)
    gsp, gf, gx0 = eng.adjoint(to_dev(target))
    torch.cuda.synchronize()
    out = [t.cpu().numpy().astype(np.float64) for t in (x, gsp, gf, gx0)]
    eng.close()
    return out


@pytest.mark.parametrize("shape,radii,sig,K,ckpt", [
    ((6, 20, 30), (1, 2, 2), (1.0, 1.5, 1.5), 5, 8),      # generic kernel, one segment
    ((8, 32, 32), (2, 5, 5), (1.5, 3.0, 3.0), 11, 4),     # specialised kernel, 3 segments
    ((5, 17, 130), (2, 4, 4), (1.5, 2.5, 2.5), 8, 8),     # specialised, ragged tiles
])
def test_adjoint_matches_oracle(cuda_device, shape, radii, sig, K, ckpt):
    rng = np.random.default_rng(sum(shape) + K)
    sp = (0.5 + 0.5 * rng.random(shape)).astype(np.float32)
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32) + 0.1
    target = (rng.random(shape) > 0.5).astype(np.float32)
    x, gsp, gf, gx0 = _gpu_grads(sp, f, x0, K, radii, sig, 1.0, target, ckpt)
    r_x0, r_sp, r_f, fw = oracle.adjoint(sp, f, x0, K, radii, sig, 1.0, target)
    assert rel_l2(x, fw["x"]) < 1e-5
    assert rel_l2(gx0, r_x0) < TOL_ADJ
    assert rel_l2(gsp, r_sp) < TOL_ADJ
    assert rel_l2(gf, r_f) < TOL_ADJ


def test_adjoint_scale_invariance(cuda_device):
    """x^K does not depend on the scale of x0, so x0 . dL/dx0 = 0."""
    rng = np.random.default_rng(41)
    shape = (6, 24, 40)
    sp = (0.5 + 0.5 * rng.random(shape)).astype(np.float32)
    f = rng.random(shape, dtype=np.float32)
    x0 = rng.random(shape, dtype=np.float32)
    _, _, _, gx0 = _gpu_grads(sp, f, x0, 6, (2, 5, 5), (1.5, 3, 3), 1.0,
                              rng.random(shape).astype(np.float32))
    assert abs(np.vdot(x0, gx0)) < 1e-5 * np.linalg.norm(x0) * np.linalg.norm(gx0)


def test_autograd_chain_through_pow(cuda_device):
    """SFSegPower inside torch autograd with sp = f^p and S = F = f: the
    gradient w.r.t. f and x0 matches the oracle's (chain rule by hand)."""
    import torch
    rng = np.random.default_rng(42)
    shape, radii, sig, K, p = (8, 32, 32), (2, 5, 5), (1.5, 3.0, 3.0), 7, 1.0
    f_np = (0.2 + 0.8 * rng.random(shape)).astype(np.float32)
    x0_np = f_np.copy()
    target = (rng.random(shape) > 0.7).astype(np.float32)
    f = to_dev(f_np).requires_grad_(True)
    x0 = to_dev(x0_np).requires_grad_(True)
    eng = make_engine(shape, radii=radii, sigmas=sig, alpha=1.0, p=p)
    x = SFSegPower.apply(f ** p, f, x0, eng, K)
    loss = (x * to_dev(target)).sum()
    loss.backward()
    torch.cuda.synchronize()
    r_x0, r_sp, r_f, _ = oracle.adjoint(f_np.astype(np.float64) ** p, f_np, x0_np, K, radii, sig,
                                        1.0, target)
    r_df = p * f_np.astype(np.float64) ** (p - 1) * r_sp + r_f
    assert rel_l2(f.grad.cpu().numpy(), r_df) < TOL_ADJ
    assert rel_l2(x0.grad.cpu().numpy(), r_x0) < TOL_ADJ
    eng.close()


def test_adjoint_needs_recorded_forward(cuda_device):
    import torch
    eng = sf.SFSeg((2, 8, 8), radii=(1, 1, 1), sigmas=(1, 1, 1))
    with pytest.raises(sf.SFSegError) as ei:
        eng.adjoint(torch.zeros((2, 8, 8), device="cuda"))
    assert ei.value.status == sf.SFSEG_ESTATE
    eng.close()


def test_adjoint_fullsize_directional_derivative(cuda_device):
    """48 x 480 x 854, 40 steps, checkpoints every 8: the adjoint's
    directional derivative along a random direction of x0 and of f matches a
    central finite difference of the FP32 forward (loose: FP32 forward), and
    x0 . dL/dx0 = 0."""
    import torch
    wl = inputs.WORKLOADS["grad_48x480x854"]
    f_np, mask = inputs.workload_video(wl.name)
    f_np = np.clip(f_np, 0.05, 1.0).astype(np.float32)
    shape, radii, sig = f_np.shape, (wl.rt, wl.ry, wl.rx), (wl.sigma_t, wl.sigma_xy, wl.sigma_xy)
    eng = make_engine(shape, radii=radii, sigmas=sig, alpha=wl.alpha, p=wl.p)
    d_f = to_dev(f_np)
    target = to_dev(mask.astype(np.float32))
    x = eng.power_iterate(d_f, d_f, d_f, wl.iters)
    gsp, gf, gx0 = eng.adjoint(target)
    rng = np.random.default_rng(43)
    v = to_dev(rng.standard_normal(shape).astype(np.float32))

    def L(sp_, f_, x0_):
        e2 = sf.SFSeg(shape, radii=radii, sigmas=sig, alpha=wl.alpha, p=wl.p, flags=sf.SFSEG_S_IS_SP)
        xx = e2.power_iterate(sp_, f_, x0_, wl.iters)
        val = float((xx.double() * target.double()).sum())
        e2.close()
        return val

    h = 1e-2
    fd_x0 = (L(d_f, d_f, d_f + h * v) - L(d_f, d_f, d_f - h * v)) / (2 * h)
    an_x0 = float((gx0.double() * v.double()).sum())
    assert abs(fd_x0 - an_x0) <= 2e-2 * max(abs(an_x0), 1e-6 * float(gx0.norm() * v.norm()))
    fd_sp = (L(d_f + h * v, d_f, d_f) - L(d_f - h * v, d_f, d_f)) / (2 * h)
    an_sp = float((gsp.double() * v.double()).sum())
    assert abs(fd_sp - an_sp) <= 2e-2 * abs(an_sp)
    assert abs(float((d_f.double() * gx0.double()).sum())) < 1e-4 * float(d_f.norm() * gx0.norm())
    eng.close()
