"""GB300-native SFSeg power iteration (arXiv 1907.02731), Python binding.

The compute lives in ``libsfseg.so`` (hand-written sm_103a CUDA behind the
C-ABI of ``include/sfseg.h``).  This module only marshals arguments: the
``sfseg_*`` functions mirror the C entry points one to one and take raw
device pointers (ints) and a ``cudaStream_t`` (int, 0 = default stream).
``SFSeg`` is a small convenience wrapper for torch CUDA tensors; torch is
used for device memory and streams only.

There is no CPU fallback: if the library is not built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

from . import inputs  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
# SFSEG_LIBRARY=debug selects the bounds-checked build (libsfseg_debug.so)
LIB_PATH = os.path.join(_HERE, "_build", "libsfseg_debug.so" if os.environ.get("SFSEG_LIBRARY") == "debug"
                        else "libsfseg.so")

SFSEG_OK, SFSEG_EINVAL, SFSEG_ENOMEM, SFSEG_ECUDA, SFSEG_EZERONORM = 0, 1, 2, 3, 4
SFSEG_ENONFINITE, SFSEG_ETIMEOUT, SFSEG_EUNSUPPORTED, SFSEG_ESTATE = 5, 6, 7, 8
SFSEG_F32, SFSEG_BF16, SFSEG_F16 = 0, 1, 2
SFSEG_S_IS_SP, SFSEG_NO_GRAPH, SFSEG_RECORD, SFSEG_GENERIC = 1, 2, 4, 8
SFSEG_FUSED, SFSEG_AUTOTUNE, SFSEG_CLUSTER = 16, 32, 64
SFSEG_PATH_FAST, SFSEG_PATH_GENERIC, SFSEG_PATH_FUSED, SFSEG_PATH_CLUSTER = 0, 1, 2, 3
PATH_NAMES = {SFSEG_PATH_FAST: "fast", SFSEG_PATH_GENERIC: "generic", SFSEG_PATH_FUSED: "fused",
              SFSEG_PATH_CLUSTER: "cluster"}
STORAGE = {"f32": SFSEG_F32, "bf16": SFSEG_BF16, "f16": SFSEG_F16}

# Every entry point declared in include/sfseg.h.
EXPORTS = (
    "sfseg_default_params", "sfseg_create", "sfseg_create_batched", "sfseg_destroy",
    "sfseg_load_features", "sfseg_power_iterate", "sfseg_load_features_batched",
    "sfseg_power_iterate_batched", "sfseg_rayleigh", "sfseg_apply", "sfseg_get_trace",
    "sfseg_adjoint", "sfseg_sync_status", "sfseg_last_error", "sfseg_status_string",
    "sfseg_launch_count", "sfseg_power_iterate_noalloc", "sfseg_plan_segments",
    "sfseg_default_binarize", "sfseg_power_iterate_binarized", "sfseg_debug_inject_timeout",
    "sfseg_get_warnings", "sfseg_get_path", "sfseg_create_slab", "sfseg_slab_start",
    "sfseg_slab_set_norm", "sfseg_slab_step", "sfseg_slab_finish_step", "sfseg_slab_halo",
    "sfseg_slab_halo_bytes", "sfseg_slab_output", "sfseg_debug_build", "sfseg_debug_status",
)
SFSEG_WARN_NEGATIVE_M = 1


class sfseg_binarize(ctypes.Structure):
    """Binarisation schedule (Alg. 1 Step 3): projection after steps k0.. of
    p = sigmoid(beta (x / max x - tau)), final mask x >= theta max x."""
    _fields_ = [("k0", ctypes.c_int32), ("reserved", ctypes.c_int32), ("beta", ctypes.c_double),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double)]


class sfseg_params(ctypes.Structure):
    _fields_ = [("nf", ctypes.c_int32), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("rt", ctypes.c_int32), ("ry", ctypes.c_int32), ("rx", ctypes.c_int32),
                ("sigma_t", ctypes.c_double), ("sigma_y", ctypes.c_double),
                ("sigma_x", ctypes.c_double), ("alpha", ctypes.c_double), ("p", ctypes.c_double),
                ("storage", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("nchan", ctypes.c_int32), ("ckpt_every", ctypes.c_int32)]


class SFSegError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


_LIB = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_pp = ctypes.POINTER(ctypes.c_void_p)


def load_library(path: str = LIB_PATH):
    """Load libsfseg.so (built by ``__graft_entry__.build()`` or ``build.py``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run `python -m paper_1907_02731_gb300.build`")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(sfseg_params)
    sig = {
        "sfseg_default_params": (None, [P, _i32, _i32, _i32]),
        "sfseg_create": (_i32, [P, ctypes.POINTER(_vp)]),
        "sfseg_create_batched": (_i32, [P, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_vp)]),
        "sfseg_destroy": (None, [_vp]),
        "sfseg_load_features": (_i32, [_vp, _vp, _vp, _vp]),
        "sfseg_power_iterate": (_i32, [_vp, _vp, _vp, _vp, _i32, _dbl, ctypes.POINTER(_i32), _vp]),
        "sfseg_load_features_batched": (_i32, [_vp, _pp, _pp, _vp]),
        "sfseg_power_iterate_batched": (_i32, [_vp, _pp, _pp, _pp, _i32, _vp]),
        "sfseg_rayleigh": (_i32, [_vp, _vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _vp]),
        "sfseg_apply": (_i32, [_vp, _vp, _vp, _vp]),
        "sfseg_get_trace": (_i32, [_vp, _i32, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl),
                                   ctypes.POINTER(_dbl), _i32]),
        "sfseg_adjoint": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
        "sfseg_sync_status": (_i32, [_vp]),
        "sfseg_last_error": (ctypes.c_char_p, [_vp]),
        "sfseg_status_string": (ctypes.c_char_p, [_i32]),
        "sfseg_launch_count": (ctypes.c_int64, [_vp]),
        "sfseg_power_iterate_noalloc": (_i32, [P, _vp, _vp, _vp, _i32, _vp, _vp]),
        "sfseg_plan_segments": (_i32, [_i32, ctypes.POINTER(_i32), _i32, ctypes.POINTER(_i32),
                                       _i32, ctypes.POINTER(_i32), _i32]),
        "sfseg_default_binarize": (None, [ctypes.POINTER(sfseg_binarize)]),
        "sfseg_debug_inject_timeout": (_i32, [_vp, _i32]),
        "sfseg_get_warnings": (_i32, [_vp, ctypes.POINTER(_i32)]),
        "sfseg_get_path": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_dbl)]),
        "sfseg_create_slab": (_i32, [P, _i32, _i32, ctypes.c_int64, ctypes.POINTER(_vp)]),
        "sfseg_slab_start": (_i32, [_vp, _vp, _i32, _vp, _vp]),
        "sfseg_slab_set_norm": (_i32, [_vp, _vp, _vp]),
        "sfseg_slab_step": (_i32, [_vp, _vp, _vp, _vp]),
        "sfseg_slab_finish_step": (_i32, [_vp, _vp, _vp]),
        "sfseg_slab_halo": (_i32, [_vp, _i32, _i32, _vp, _vp]),
        "sfseg_slab_halo_bytes": (ctypes.c_int64, [_vp, _i32, _i32]),
        "sfseg_slab_output": (_i32, [_vp, _vp, _vp]),
        "sfseg_debug_build": (_i32, []),
        "sfseg_debug_status": (_i32, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_i32),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "sfseg_power_iterate_binarized": (_i32, [_vp, _vp, _vp, _vp, _i32,
                                                 ctypes.POINTER(sfseg_binarize), _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _status_name(st: int) -> str:
    names = {0: "SFSEG_OK", 1: "SFSEG_EINVAL", 2: "SFSEG_ENOMEM", 3: "SFSEG_ECUDA",
             4: "SFSEG_EZERONORM", 5: "SFSEG_ENONFINITE", 6: "SFSEG_ETIMEOUT",
             7: "SFSEG_EUNSUPPORTED", 8: "SFSEG_ESTATE"}
    return names.get(st, f"status {st}")


def _check(st: int, ctx=None):
    if st != SFSEG_OK:
        msg = load_library().sfseg_last_error(ctx)
        raise SFSegError(st, msg.decode() if msg else "")


def _ptrs(seq):
    arr = (ctypes.c_void_p * len(seq))(*[int(p) for p in seq])
    return ctypes.cast(arr, _pp), arr


# ------------------------------------------------------- C entry points, 1:1
def sfseg_default_params(nf: int, h: int, w: int) -> sfseg_params:
    p = sfseg_params()
    load_library().sfseg_default_params(ctypes.byref(p), nf, h, w)
    return p


def sfseg_create(params: sfseg_params) -> int:
    out = _vp()
    _check(load_library().sfseg_create(ctypes.byref(params), ctypes.byref(out)))
    return out.value


def sfseg_create_batched(params: sfseg_params, dims) -> int:
    flat = (_i32 * (3 * len(dims)))(*[int(v) for d in dims for v in d])
    out = _vp()
    _check(load_library().sfseg_create_batched(ctypes.byref(params), len(dims), flat,
                                               ctypes.byref(out)))
    return out.value


def sfseg_destroy(ctx: int) -> None:
    load_library().sfseg_destroy(ctx)


def sfseg_load_features(ctx: int, d_s: int, d_f: int, stream: int = 0) -> None:
    _check(load_library().sfseg_load_features(ctx, d_s, d_f, stream), ctx)


def sfseg_power_iterate(ctx: int, d_s, d_f, d_x: int, n_iters: int, tol: float = 0.0,
                        want_iters_done: bool = False, stream: int = 0):
    done = _i32(-1)
    st = load_library().sfseg_power_iterate(ctx, d_s, d_f, d_x, n_iters, tol,
                                            ctypes.byref(done) if want_iters_done else None, stream)
    _check(st, ctx)
    return done.value if want_iters_done else None


def sfseg_load_features_batched(ctx: int, d_s, d_f, stream: int = 0) -> None:
    ps, ks = _ptrs(d_s)
    pf, kf = _ptrs(d_f)
    _check(load_library().sfseg_load_features_batched(ctx, ps, pf, stream), ctx)


def sfseg_power_iterate_batched(ctx: int, d_s, d_f, d_x, n_iters: int, stream: int = 0) -> None:
    px, kx = _ptrs(d_x)
    if d_s is None:
        _check(load_library().sfseg_power_iterate_batched(ctx, None, None, px, n_iters, stream), ctx)
        return
    ps, ks = _ptrs(d_s)
    pf, kf = _ptrs(d_f)
    _check(load_library().sfseg_power_iterate_batched(ctx, ps, pf, px, n_iters, stream), ctx)


def sfseg_rayleigh(ctx: int, d_x: int, stream: int = 0):
    lam, res = _dbl(), _dbl()
    _check(load_library().sfseg_rayleigh(ctx, d_x, ctypes.byref(lam), ctypes.byref(res), stream), ctx)
    return lam.value, res.value


def sfseg_apply(ctx: int, d_x: int, d_y: int, stream: int = 0) -> None:
    _check(load_library().sfseg_apply(ctx, d_x, d_y, stream), ctx)


def sfseg_get_trace(ctx: int, video: int = 0, cap: int = 100000):
    import numpy as np
    r, rho, nrm = (np.zeros(cap) for _ in range(3))
    P = ctypes.POINTER(_dbl)
    n = load_library().sfseg_get_trace(ctx, video, r.ctypes.data_as(P), rho.ctypes.data_as(P),
                                       nrm.ctypes.data_as(P), cap)
    if n < 0:
        _check(SFSEG_ECUDA, ctx)
    return dict(rayleigh=r[:n], residual=rho[:n], norms=nrm[:n])


def sfseg_adjoint(ctx: int, d_gx: int, d_gsp, d_gf, d_gx0, stream: int = 0) -> None:
    _check(load_library().sfseg_adjoint(ctx, d_gx, d_gsp, d_gf, d_gx0, stream), ctx)


def sfseg_sync_status(ctx: int) -> int:
    return load_library().sfseg_sync_status(ctx)


def sfseg_last_error(ctx) -> str:
    m = load_library().sfseg_last_error(ctx)
    return m.decode() if m else ""


def sfseg_status_string(st: int) -> str:
    return load_library().sfseg_status_string(st).decode()


def sfseg_launch_count(ctx: int) -> int:
    return int(load_library().sfseg_launch_count(ctx))


def sfseg_power_iterate_noalloc(params: sfseg_params, d_s: int, d_f: int, d_x: int,
                                n_iters: int, d_trace=None, stream: int = 0) -> None:
    """Allocation-free power iteration (fixed workspace inside the library);
    for callers that may not call cudaMalloc.  See include/sfseg.h."""
    _check(load_library().sfseg_power_iterate_noalloc(ctypes.byref(params), d_s, d_f, d_x,
                                                      n_iters, d_trace, stream))


def sfseg_default_binarize() -> sfseg_binarize:
    b = sfseg_binarize()
    load_library().sfseg_default_binarize(ctypes.byref(b))
    return b


def sfseg_power_iterate_binarized(ctx, d_s, d_f, d_x, n_iters: int, b: sfseg_binarize,
                                  d_mask=None, stream: int = 0) -> None:
    _check(load_library().sfseg_power_iterate_binarized(ctx, d_s, d_f, d_x, n_iters, ctypes.byref(b),
                                                        d_mask, stream), ctx)


def sfseg_plan_segments(dims, n_sms: int):
    """Work decomposition of the specialised kernel (host only): returns
    (segments [n][5] as (video, x0, y0, t0, t1), cta_begin list)."""
    flat = (_i32 * (3 * len(dims)))(*[int(v) for d in dims for v in d])
    L = load_library()
    n = L.sfseg_plan_segments(len(dims), flat, n_sms, None, 0, None, 0)
    if n < 0:
        _check(SFSEG_EINVAL)
    segs = (_i32 * (5 * n))()
    cb = (_i32 * (n_sms + 1))(*([-1] * (n_sms + 1)))
    L.sfseg_plan_segments(len(dims), flat, n_sms, segs, n, cb, n_sms + 1)
    rows = [tuple(segs[5 * i:5 * i + 5]) for i in range(n)]
    cta = [c for c in cb if c >= 0]
    return rows, cta


def sfseg_get_path(ctx: int):
    """(path, fused CTA count, [us per step measured per path or -1]) of a context."""
    path, ctas, us = _i32(), _i32(), (_dbl * 4)()
    _check(load_library().sfseg_get_path(ctx, ctypes.byref(path), ctypes.byref(ctas), us), ctx)
    return path.value, ctas.value, list(us)


def sfseg_create_slab(params: sfseg_params, own_lo: int, own_hi: int, video_voxels: int) -> int:
    out = _vp()
    _check(load_library().sfseg_create_slab(ctypes.byref(params), own_lo, own_hi, video_voxels,
                                            ctypes.byref(out)))
    return out.value


def sfseg_slab_start(ctx: int, d_x0: int, n_iters: int, d_part: int, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_start(ctx, d_x0, n_iters, d_part, stream), ctx)


def sfseg_slab_set_norm(ctx: int, d_sumsq: int, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_set_norm(ctx, d_sumsq, stream), ctx)


def sfseg_slab_step(ctx: int, d_part: int, d_x_final=None, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_step(ctx, d_part, d_x_final, stream), ctx)


def sfseg_slab_finish_step(ctx: int, d_sums: int, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_finish_step(ctx, d_sums, stream), ctx)


def sfseg_slab_halo(ctx: int, side: int, direction: int, d_buf: int, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_halo(ctx, side, direction, d_buf, stream), ctx)


def sfseg_slab_halo_bytes(ctx: int, side: int, direction: int) -> int:
    n = load_library().sfseg_slab_halo_bytes(ctx, side, direction)
    if n < 0:
        _check(SFSEG_EINVAL, ctx)
    return n


def sfseg_slab_output(ctx: int, d_x: int, stream: int = 0) -> None:
    _check(load_library().sfseg_slab_output(ctx, d_x, stream), ctx)


def sfseg_debug_status():
    """(violations, first code, first values) of the bounds-checked build since
    the last call (zeros in the normal build); synchronises the device."""
    n, code, a, b = ctypes.c_int64(), _i32(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().sfseg_debug_status(ctypes.byref(n), ctypes.byref(code), ctypes.byref(a),
                                             ctypes.byref(b)))
    return n.value, code.value, (a.value, b.value)


# --------------------------------------------------- torch convenience wrapper
def _stream_handle():
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def _dev_f32(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


class SFSeg:
    """One context for volumes of shape (nf, h, w) (or a batch of shapes).

    ``radii`` = (rt, ry, rx), ``sigmas`` = (sigma_t, sigma_y, sigma_x);
    ``nchan`` > 1 sums the affinities of several pairwise feature channels
    (Eq. 9), ``f`` then being a contiguous [nchan, nf, h, w] tensor.
    """

    def __init__(self, shape=None, *, radii=(2, 5, 5), sigmas=(1.5, 3.0, 3.0), alpha=1.0,
                 p=0.1, storage="f32", flags=0, batch_shapes=None, ckpt_every=8, nchan=1):
        nf, h, w = shape if shape is not None else (1, 1, 1)
        prm = sfseg_default_params(nf, h, w)
        prm.rt, prm.ry, prm.rx = radii
        prm.sigma_t, prm.sigma_y, prm.sigma_x = sigmas
        prm.alpha, prm.p = alpha, p
        prm.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        prm.flags = flags
        prm.ckpt_every = ckpt_every
        prm.nchan = nchan              # Eq. 9 channels: f is then [nchan, nf, h, w]
        self.params = prm
        self.batch_shapes = [tuple(s) for s in batch_shapes] if batch_shapes else None
        self.shape = tuple(shape) if shape is not None else None
        self.ctx = (sfseg_create_batched(prm, self.batch_shapes) if self.batch_shapes
                    else sfseg_create(prm))

    def close(self):
        if getattr(self, "ctx", None):
            sfseg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_features(self, s, f):
        sfseg_load_features(self.ctx, _dev_f32(s, "s").data_ptr(), _dev_f32(f, "f").data_ptr(),
                            _stream_handle())

    def power_iterate(self, s, f, x0, iters: int, tol: float = 0.0, out=None):
        """x^K from x0 (a new tensor unless ``out`` is given; x0 is not modified)."""
        import torch
        x = out if out is not None else torch.empty_like(_dev_f32(x0, "x0"))
        if x.data_ptr() != x0.data_ptr():
            x.copy_(x0)
        ds = _dev_f32(s, "s").data_ptr() if s is not None else None
        df = _dev_f32(f, "f").data_ptr() if f is not None else None
        self.iters_done = sfseg_power_iterate(self.ctx, ds, df, _dev_f32(x, "x").data_ptr(), iters,
                                              tol, want_iters_done=tol > 0, stream=_stream_handle())
        return x

    def power_iterate_binarized(self, s, f, x0, iters: int, k0: int = 3, beta: float = 10.0,
                                tau: float = 0.5, theta: float = 0.5, out=None):
        """x^K with the binarisation schedule of Alg. 1 (sigmoid projections
        after steps k0..K-1) and the hard mask x^K >= theta max(x^K) (uint8)."""
        import torch
        x = out if out is not None else torch.empty_like(_dev_f32(x0, "x0"))
        if x.data_ptr() != x0.data_ptr():
            x.copy_(x0)
        mask = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
        b = sfseg_binarize(k0=k0, reserved=0, beta=beta, tau=tau, theta=theta)
        ds = _dev_f32(s, "s").data_ptr() if s is not None else None
        df = _dev_f32(f, "f").data_ptr() if f is not None else None
        sfseg_power_iterate_binarized(self.ctx, ds, df, _dev_f32(x, "x").data_ptr(), iters, b,
                                      mask.data_ptr(), _stream_handle())
        return x, mask

    def warnings(self) -> int:
        """Bits of SFSEG_WARN_* about the loaded features (synchronises)."""
        fl = _i32(0)
        _check(load_library().sfseg_get_warnings(self.ctx, ctypes.byref(fl)), self.ctx)
        return int(fl.value)

    def debug_inject_timeout(self, n_steps: int = 1):
        """Test aid: the next n_steps steps give up on a device-side wait and
        report SFSEG_ETIMEOUT (see include/sfseg.h)."""
        _check(load_library().sfseg_debug_inject_timeout(self.ctx, n_steps), self.ctx)

    def power_iterate_batched(self, s_list, f_list, x_list, iters: int):
        """In place on ``x_list`` (x0 in, x^K out)."""
        ds = [_dev_f32(t, "s").data_ptr() for t in s_list] if s_list is not None else None
        df = [_dev_f32(t, "f").data_ptr() for t in f_list] if f_list is not None else None
        dx = [_dev_f32(t, "x").data_ptr() for t in x_list]
        sfseg_power_iterate_batched(self.ctx, ds, df, dx, iters, _stream_handle())
        return x_list

    def rayleigh(self, x):
        return sfseg_rayleigh(self.ctx, _dev_f32(x, "x").data_ptr(), _stream_handle())

    def apply(self, x, out=None):
        import torch
        y = out if out is not None else torch.empty_like(_dev_f32(x, "x"))
        sfseg_apply(self.ctx, x.data_ptr(), _dev_f32(y, "y").data_ptr(), _stream_handle())
        return y

    def adjoint(self, gx):
        """(dL/dsp, dL/df, dL/dx0) of the last recorded power_iterate, given
        dL/dx^K (the context must be created with SFSEG_RECORD)."""
        import torch
        gx = _dev_f32(gx, "gx")
        gsp, gf, gx0 = (torch.empty_like(gx) for _ in range(3))
        sfseg_adjoint(self.ctx, gx.data_ptr(), gsp.data_ptr(), gf.data_ptr(), gx0.data_ptr(),
                      _stream_handle())
        return gsp, gf, gx0

    def trace(self, video: int = 0):
        return sfseg_get_trace(self.ctx, video)

    def sync_status(self) -> int:
        return sfseg_sync_status(self.ctx)

    def launch_count(self) -> int:
        return sfseg_launch_count(self.ctx)

    def path(self):
        """{'path': 'fast'|'generic'|'fused'|'cluster', 'fused_ctas': n (CTAs of the fused or
        cluster launch), 'tuned_us': {...}}."""
        pth, ctas, us = sfseg_get_path(self.ctx)
        return {"path": PATH_NAMES[pth], "fused_ctas": ctas,
                "tuned_us": {PATH_NAMES[i]: u for i, u in enumerate(us) if u >= 0}}
