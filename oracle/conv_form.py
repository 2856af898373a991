"""Eq. 7 evaluated literally, with FP64 direct 3D convolutions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  This is a second,
independent routine of the oracle: it never builds M and never visits edges.
It exists to check that the convolution form (Eq. 7) equals the explicit
power-iteration step (Eq. 4) -- the identity the paper derives through
Eq. 5 and Eq. 6.  The convolution is ``scipy.ndimage.correlate`` with the full
(non-separable) 3D Gaussian and zero padding; G is symmetric, so correlation
and convolution coincide.

Eq. 7 lacks the leading alpha of Eq. 6; the routine multiplies Eq. 7 by alpha
so it returns M x of Eq. 2 (alpha * alpha^-1 is written as 1, which also
covers alpha = 0).  With channels (Eq. 9) the result is summed over them.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def gaussian_3d(gt, gy, gx) -> np.ndarray:
    """G_3D[dt, dy, dx] = g_t(dt) g_y(dy) g_x(dx)."""
    gt, gy, gx = (np.asarray(v, np.float64) for v in (gt, gy, gx))
    return gt[:, None, None] * gy[None, :, None] * gx[None, None, :]


def conv3d(v, G3) -> np.ndarray:
    """G_3D * v, 'same' size, zero padding outside the volume."""
    return ndimage.correlate(np.asarray(v, np.float64), G3, mode="constant", cval=0.0)


def apply_conv_form(sp, f, x, gt, gy, gx, alpha: float) -> np.ndarray:
    """alpha * X_crt of Eq. 7 (summed over channels for ``f`` of shape [C,...]):

      X_crt = S^p (1/alpha - F^2) G*(S^p X) - S^p G*(F^2 S^p X) + 2 S^p F G*(F S^p X)
    """
    sp = np.asarray(sp, np.float64)
    x = np.asarray(x, np.float64)
    f = np.asarray(f, np.float64)
    chans = [f] if f.ndim == 3 else list(f)
    G3 = gaussian_3d(gt, gy, gx)
    a = sp * x                                   # S^p . X^k
    conv_a = conv3d(a, G3)                       # G * (S^p X)
    out = np.zeros_like(x)
    for F in chans:
        t1 = sp * (1.0 - alpha * F * F) * conv_a          # alpha * S^p (1/alpha - F^2) G*(S^p X)
        t2 = -alpha * sp * conv3d(F * F * a, G3)          # -alpha * S^p G*(F^2 S^p X)
        t3 = 2.0 * alpha * sp * F * conv3d(F * a, G3)     # 2 alpha * S^p F G*(F S^p X)
        out += t1 + t2 + t3
    return out
