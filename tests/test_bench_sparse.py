"""The explicit-matrix comparison of the runtime sweep (Fig. 2) builds the
matrix of Eq. 2: checked entry by entry against the oracle's brute-force
dense matrix, and its product against the oracle's Eq. 2 evaluation."""
import numpy as np
import pytest

import oracle
from oracle import dense


@pytest.mark.parametrize("shape,radii,sig,alpha", [
    ((3, 5, 6), (1, 2, 2), (1.0, 1.5, 2.0), 1.0),
    ((4, 3, 7), (2, 1, 3), (1.5, 1.0, 3.0), 0.4),
    ((1, 4, 4), (2, 5, 5), (1.5, 3.0, 3.0), 1.0),   # box wider than the volume
])
def test_explicit_matrix_is_eq2(shape, radii, sig, alpha):
    import torch
    import bench
    rng = np.random.default_rng(11)
    f = rng.random(shape).astype(np.float32)
    sp = (f.astype(np.float64) ** 0.5).astype(np.float32)
    A = bench.explicit_eq2_matrix(torch.from_numpy(sp), torch.from_numpy(f), radii, sig, alpha)
    D = dense.dense_M(sp.astype(np.float64), f.astype(np.float64),
                      *(oracle.taps(r, s) for r, s in zip(radii, sig)), alpha)
    np.testing.assert_allclose(A.to_dense().numpy(), D, rtol=1e-5, atol=1e-6)
    x = rng.random(shape)
    y = oracle.apply_M(sp.astype(np.float64), f.astype(np.float64), x, radii, sig, alpha)
    ya = (A.to_dense().double() @ torch.from_numpy(x.ravel())).numpy()
    np.testing.assert_allclose(ya, y.ravel(), rtol=1e-5, atol=1e-6)
