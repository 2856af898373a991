"""Brute-force dense adjacency for tiny volumes (N up to a few thousand).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Builds the N x N
matrix of Eq. 2 (or Eq. 1) by comparing every pair of voxel coordinates, so
that the dense FP64 eigendecomposition (LAPACK ``eigh``) can stand in for the
"standard routine" the paper compares against (Sec. 4, Fig. 3).
"""
from __future__ import annotations

import numpy as np


def dense_M(sp, f, gt, gy, gx, alpha: float, exact: bool = False) -> np.ndarray:
    sp = np.asarray(sp, np.float64)
    f = np.asarray(f, np.float64)
    nf, h, w = sp.shape
    rt, ry, rx = (len(g) // 2 for g in (gt, gy, gx))
    t, y, x = np.meshgrid(np.arange(nf), np.arange(h), np.arange(w), indexing="ij")
    t, y, x = t.ravel(), y.ravel(), x.ravel()
    dt = t[:, None] - t[None, :]
    dy = y[:, None] - y[None, :]
    dx = x[:, None] - x[None, :]
    inside = (np.abs(dt) <= rt) & (np.abs(dy) <= ry) & (np.abs(dx) <= rx)
    gt, gy, gx = (np.asarray(g, np.float64) for g in (gt, gy, gx))
    G = np.where(inside,
                 gt[np.clip(dt + rt, 0, 2 * rt)] * gy[np.clip(dy + ry, 0, 2 * ry)]
                 * gx[np.clip(dx + rx, 0, 2 * rx)], 0.0)
    s = sp.ravel()
    fv = f.ravel()
    d = fv[:, None] - fv[None, :]
    pair = np.exp(-alpha * d * d) if exact else 1.0 - alpha * d * d
    return s[:, None] * s[None, :] * pair * G


def principal_eigvec(M) -> tuple[float, np.ndarray]:
    """Largest eigenvalue and its unit eigenvector, oriented to sum >= 0."""
    vals, vecs = np.linalg.eigh(M)
    v = vecs[:, -1]
    if v.sum() < 0:
        v = -v
    return float(vals[-1]), v
