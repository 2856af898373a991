"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding, run the oracle on the same seeded inputs, compare."""
import numpy as np

import oracle
import paper_1907_02731_gb300 as sf

# FP32 bar for eigenvector iterates and one-step outputs against the FP64
# oracle (relative L2), and the BF16/FP16-storage bar.
TOL_F32 = 1e-5
TOL_LOWP = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def gpu_power(f, x0, K, radii, sigmas, alpha, p, s=None, storage="f32", flags=0, tol=0.0):
    """x^K and the trace from the CUDA path (C-ABI through the binding)."""
    import torch
    s = f if s is None else s
    eng = sf.SFSeg(f.shape, radii=radii, sigmas=sigmas, alpha=alpha, p=p, storage=storage,
                   flags=flags)
    try:
        x = to_dev(x0)
        try:
            eng.power_iterate(to_dev(s), to_dev(f), x, K, tol=tol, out=x)
        except sf.SFSegError as e:      # device-side status reported by a synchronising call
            if e.status not in (sf.SFSEG_EZERONORM, sf.SFSEG_ENONFINITE):
                raise
        torch.cuda.synchronize()
        tr = eng.trace()
        st = eng.sync_status()
        return x.cpu().numpy(), tr, st, len(tr["rayleigh"])
    finally:
        eng.close()


def oracle_power(f, x0, K, radii, sigmas, alpha, p, s=None, storage="f32"):
    """The FP64 oracle on the same inputs; with a low-precision storage type
    it ingests the same rounded sp, f, x0 the kernel sees."""
    s = f if s is None else s
    sp = oracle.unary(np.asarray(s, np.float64), p)
    if storage != "f32":
        sp = oracle.to_storage(np.asarray(s, np.float32) ** np.float32(p), storage)
        f64 = oracle.to_storage(f, storage)
        x064 = oracle.to_storage(x0, storage)
    else:
        f64 = np.asarray(f, np.float64)
        x064 = np.asarray(x0, np.float64)
    return oracle.power_iterate(sp, f64, x064, K, radii, sigmas, alpha)
