"""Algorithm 1 with its binarisation step -- TEST INFRASTRUCTURE ONLY.

FP64 CPU restatement of Step 3 of Algorithm 1 and of Sec. 4 ("Binarization -
Spectral vs Discrete space"): the power iteration runs in the continuous space
for a few steps; from then on, after each step, the iterate is projected
through a sigmoid onto an almost discrete space and the next step starts from
the projection; after the last step a hard threshold gives the segmentation.

The paper gives none of the values.  Reading used here (and by the library):
with u = x / max(x) (x >= 0 by Perron-Frobenius, u in [0, 1]),
    after step j (1-based), k0 <= j < K:   p = 1 / (1 + exp(-beta (u - tau))),
                                           x = p / ||p||;
    after the last step:                   mask = [u >= theta].
The mask decision is taken in FP32 (x and theta * max(x) rounded to FP32),
the precision of the CUDA path's compare.  Each power step is the oracle's
edge-by-edge y = M x (Eq. 2, Eq. 4), then x = y / ||y|| (Eq. 8).
"""
from __future__ import annotations

import numpy as np

from . import apply_M


def power_iterate_binarized(sp, f, x0, K: int, radii, sigmas, alpha: float, k0: int,
                            beta: float, tau: float, theta: float) -> dict:
    """x^K, the hard mask and the Rayleigh quotients r_k = x^k.Mx^k / x^k.x^k."""
    x = np.asarray(x0, np.float64)
    x = x / np.linalg.norm(x)
    rayleigh = []
    for k in range(K):
        y = apply_M(sp, f, x, radii, sigmas, alpha)                 # Step 2: y = M x
        rayleigh.append(float(np.vdot(x, y) / np.vdot(x, x)))
        x = y / np.linalg.norm(y)                                    # normalise
        j = k + 1                                                    # steps done
        if k0 <= j < K:                                              # Step 3: project
            u = x / x.max()
            p = 1.0 / (1.0 + np.exp(-beta * (u - tau)))
            x = p / np.linalg.norm(p)
    x32 = x.astype(np.float32)
    cut = np.float32(theta) * x32.max()
    return {"x": x, "mask": (x32 >= cut).astype(np.uint8), "rayleigh": np.asarray(rayleigh)}
