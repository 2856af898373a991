"""FP64 CPU oracle for the SFSeg power iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1907_02731_gb300``) and never imports it.

Contents
  * ``sfseg_oracle.c`` (loaded here through ctypes): the explicit, edge-by-edge
    definition -- M_ij of Eq. 2 (or Eq. 1 with ``mode=1``), y = M x of Eq. 4,
    the normalised power iteration of Eq. 8 / Algorithm 1 with the Rayleigh
    quotient of Eq. 3, and the reverse-mode derivative of the unrolled
    iteration.
  * ``conv_form.py``: a second, independent FP64 routine that evaluates the
    3D-convolution form of Eq. 7 with direct (non-separable) convolutions; it
    exists to check Eq. 4 == Eq. 7 and is used by that test only.
  * ``dense.py``: brute-force dense M for tiny volumes (eigendecomposition).
  * ``binarize.py``: Algorithm 1 with the binarisation step (sigmoid
    projections, final hard threshold) on top of the edge-by-edge M.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, special cases, dense eigendecomposition, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfseg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, FP64, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        geo = [_i64, _i64, _i64, _int, _int, _int, _dp, _dp, _dp, _dbl, _int, _int, _dp, _dp]
        lib.oracle_taps.argtypes = [_int, _dbl, _dp]
        lib.oracle_unary.argtypes = [_dp, _i64, _dbl, _dp]
        lib.oracle_apply.argtypes = geo + [_dp, _dp]
        lib.oracle_apply_at.argtypes = geo + [_dp, _lp, _i64, _dp]
        lib.oracle_power.argtypes = geo + [_dp, _int, _dp, _dp, _dp, _dp, _dp, _ip]
        lib.oracle_power.restype = _int
        lib.oracle_adjoint.argtypes = [_i64, _i64, _i64, _int, _int, _int, _dp, _dp, _dp,
                                       _dbl, _dp, _dp, _dp, _dp, _int, _dp, _dp, _dp, _dp]
        _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def taps(r: int, sigma: float) -> np.ndarray:
    """Gaussian taps g(d) = exp(-d^2 / 2 sigma^2), d = -r..r (Eq. 1's G, peak 1)."""
    g = np.empty(2 * r + 1, np.float64)
    _lib().oracle_taps(int(r), float(sigma), _p(g))
    return g


def unary(s, p: float) -> np.ndarray:
    """sp = s^p (the unary term of Eq. 1)."""
    s = _f64(s)
    out = np.empty_like(s)
    _lib().oracle_unary(_p(s), s.size, float(p), _p(out))
    return out


class Geometry:
    """Volume shape and Gaussian support of one problem."""

    def __init__(self, shape, radii, sigmas):
        self.nf, self.h, self.w = (int(v) for v in shape)
        self.rt, self.ry, self.rx = (int(v) for v in radii)
        st, sy, sx = (float(v) for v in sigmas)
        self.gt, self.gy, self.gx = taps(self.rt, st), taps(self.ry, sy), taps(self.rx, sx)

    @property
    def n(self):
        return self.nf * self.h * self.w

    def args(self):
        return (self.nf, self.h, self.w, self.rt, self.ry, self.rx,
                _p(self.gt), _p(self.gy), _p(self.gx))


def _features(f, shape):
    f = _f64(f)
    nc = 1 if f.ndim == 3 else f.shape[0]
    assert f.shape[-3:] == tuple(shape)
    return f, nc


def apply_M(sp, f, x, radii, sigmas, alpha: float, mode: int = 0) -> np.ndarray:
    """y = M x with M of Eq. 2 (mode 0) or Eq. 1 (mode 1), explicit edges.

    ``f`` is ``[nf,h,w]`` or ``[C,nf,h,w]`` (Eq. 9 channels, Taylor form only).
    """
    sp, x = _f64(sp), _f64(x)
    geo = Geometry(sp.shape, radii, sigmas)
    f, nc = _features(f, sp.shape)
    y = np.empty_like(x)
    _lib().oracle_apply(*geo.args(), float(alpha), int(mode), nc, _p(sp), _p(f), _p(x), _p(y))
    return y


def apply_M_at(sp, f, x, radii, sigmas, alpha: float, idx, mode: int = 0) -> np.ndarray:
    """(M x)_i at flat indices ``idx`` only."""
    sp, x = _f64(sp), _f64(x)
    geo = Geometry(sp.shape, radii, sigmas)
    f, nc = _features(f, sp.shape)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, np.float64)
    _lib().oracle_apply_at(*geo.args(), float(alpha), int(mode), nc, _p(sp), _p(f), _p(x),
                           idx.ctypes.data_as(_lp), idx.size, _p(out))
    return out


def power_iterate(sp, f, x0, K: int, radii, sigmas, alpha: float, mode: int = 0,
                  keep: bool = False) -> dict:
    """K steps of x <- Mx / ||Mx|| from x0 (Eq. 4, Eq. 8; Algorithm 1 without
    binarisation).  Returns x (= x^K), rayleigh[k], residual[k], norms[k]
    (= ||M x^k||), k_done, status (0 ok, 1 zero norm) and, if ``keep``,
    xs = x^0..x^K."""
    sp, x0 = _f64(sp), _f64(x0)
    geo = Geometry(sp.shape, radii, sigmas)
    f, nc = _features(f, sp.shape)
    x = np.empty_like(x0)
    ray = np.zeros(K)
    res = np.zeros(K)
    nrm = np.zeros(K)
    xs = np.empty((K + 1,) + x0.shape) if keep else None
    kd = ctypes.c_int(0)
    st = _lib().oracle_power(*geo.args(), float(alpha), int(mode), nc, _p(sp), _p(f), _p(x0),
                             int(K), _p(x), _p(ray), _p(res), _p(nrm), _p(xs), ctypes.byref(kd))
    return dict(x=x, rayleigh=ray, residual=res, norms=nrm, k_done=kd.value, status=st, xs=xs)


def adjoint(sp, f, x0, K: int, radii, sigmas, alpha: float, gK):
    """Gradient of a loss with dL/dx^K = gK w.r.t. (x0, sp, f), through the
    K-step normalised iteration (single channel, Eq. 2).  Returns
    ``(g_x0, g_sp, g_f, forward_result)``."""
    sp, f, x0, gK = _f64(sp), _f64(f), _f64(x0), _f64(gK)
    fw = power_iterate(sp, f, x0, K, radii, sigmas, alpha, keep=True)
    if fw["status"] != 0:
        raise FloatingPointError("zero norm in the forward iteration")
    geo = Geometry(sp.shape, radii, sigmas)
    g_x0, g_sp, g_f = (np.empty_like(x0) for _ in range(3))
    _lib().oracle_adjoint(*geo.args(), float(alpha), _p(sp), _p(f), _p(fw["xs"]),
                          _p(fw["norms"]), int(K), _p(gK), _p(g_x0), _p(g_sp), _p(g_f))
    return g_x0, g_sp, g_f, fw


def to_storage(a, dtype: str) -> np.ndarray:
    """Round an array to a storage type ("f32", "bf16", "f16", round to
    nearest even) and return it as FP64, so the oracle sees the same input
    bytes as a low-precision run."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    if dtype == "f32":
        return a32.astype(np.float64)
    if dtype == "f16":
        return a32.astype(np.float16).astype(np.float64)
    if dtype == "bf16":
        u = a32.view(np.uint32).astype(np.uint64)
        nan = np.isnan(a32)
        rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
        out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
        out[nan] = np.nan
        return out
    raise ValueError(dtype)
