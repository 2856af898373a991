"""The C-ABI library builds, loads and exports every symbol include/sfseg.h
declares; host-side validation works without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

import paper_1907_02731_gb300 as sf
from paper_1907_02731_gb300 import build as sfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sfseg_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    sfbuild.build()
    return sf.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(sf.EXPORTS)


def test_default_params_and_status_strings(lib):
    p = sf.sfseg_default_params(72, 480, 854)
    assert (p.nf, p.h, p.w, p.rt, p.ry, p.rx) == (72, 480, 854, 2, 5, 5)
    assert (p.sigma_t, p.sigma_y, p.alpha, p.p, p.nchan) == (1.5, 3.0, 1.0, 0.1, 1)
    assert sf.sfseg_status_string(sf.SFSEG_EZERONORM) == "SFSEG_EZERONORM"
    assert sf.sfseg_status_string(99) == "SFSEG_UNKNOWN"


@pytest.mark.parametrize("field,value", [("rx", -1), ("ry", 17), ("rt", 9), ("sigma_t", 0.0),
                                         ("alpha", -1.0), ("p", float("nan")), ("storage", 3),
                                         ("nf", 0), ("w", -5), ("nchan", 0), ("flags", 128),
                                         ("flags", -1), ("flags", 16 | 8), ("flags", 16 | 32),
                                         ("flags", 64 | 8), ("flags", 64 | 16), ("flags", 64 | 32)])
def test_create_rejects_bad_params(lib, field, value):
    """Validation happens on the host before any device call."""
    p = sf.sfseg_default_params(4, 8, 8)
    setattr(p, field, value)
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_create(p)
    assert ei.value.status == sf.SFSEG_EINVAL
    assert sf.sfseg_last_error(None)


@pytest.mark.parametrize("flags,nchan", [(16 | 4, 1), (32 | 4, 1), (16, 2), (64 | 4, 1), (64, 2)])
def test_create_rejects_unsupported_paths(lib, flags, nchan):
    """The fused and cluster launches run one channel and are not recorded for
    the adjoint; the autotuner does not choose for recorded contexts (host-side
    checks)."""
    p = sf.sfseg_default_params(4, 8, 8)
    p.flags, p.nchan = flags, nchan
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_create(p)
    assert ei.value.status == sf.SFSEG_EUNSUPPORTED


def test_null_context_calls(lib):
    assert lib.sfseg_power_iterate(None, None, None, None, 1, 0.0, None, None) == sf.SFSEG_EINVAL
    assert lib.sfseg_get_trace(None, 0, None, None, None, 0) == -1
    lib.sfseg_destroy(None)
    assert lib.sfseg_launch_count(None) == 0
    assert lib.sfseg_get_path(None, None, None, None) == sf.SFSEG_EINVAL


@pytest.mark.parametrize("nchan,radii", [(5, (2, 5, 5)), (8, (1, 1, 1)), (4, (8, 16, 16)),
                                         (3, (8, 16, 16))])
def test_create_rejects_unsupported_channels(lib, nchan, radii):
    """Eq. 9 channels: at most 4, and only while the any-radius kernel's
    buffers for these radii fit in shared memory (host-side check)."""
    p = sf.sfseg_default_params(4, 8, 8)
    p.nchan = nchan
    p.rt, p.ry, p.rx = radii
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_create(p)
    assert ei.value.status == sf.SFSEG_EUNSUPPORTED
    assert "nchan" in sf.sfseg_last_error(None)


def test_noalloc_rejects_channels(lib):
    p = sf.sfseg_default_params(4, 8, 8)
    p.nchan = 2
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_power_iterate_noalloc(p, 1, 1, 1, 3)
    assert ei.value.status == sf.SFSEG_EUNSUPPORTED


def test_debug_injection_null_context(lib):
    assert lib.sfseg_debug_inject_timeout(None, 1) == sf.SFSEG_EINVAL


def test_warnings_null_arguments(lib):
    flags = ctypes.c_int32(7)
    assert lib.sfseg_get_warnings(None, ctypes.byref(flags)) == sf.SFSEG_EINVAL


def test_slab_arguments_are_checked(lib):
    """A video split along t: the slab's own range, halo and flags are
    validated on the host before any device call."""
    p = sf.sfseg_default_params(8, 16, 16)
    for lo, hi in ((3, 6), (0, 9), (2, 2), (1, 2), (-1, 4)):   # halo > rt, past the slab, empty, own < rt
        with pytest.raises(sf.SFSegError) as ei:
            sf.sfseg_create_slab(p, lo, hi, 8 * 16 * 16 * 4)
        assert ei.value.status == sf.SFSEG_EINVAL
    with pytest.raises(sf.SFSegError) as ei:
        sf.sfseg_create_slab(p, 2, 6, 10)                       # fewer video voxels than its own frames
    assert ei.value.status == sf.SFSEG_EINVAL
    for flags in (sf.SFSEG_FUSED, sf.SFSEG_AUTOTUNE, sf.SFSEG_RECORD, sf.SFSEG_CLUSTER):
        p.flags = flags
        with pytest.raises(sf.SFSegError) as ei:
            sf.sfseg_create_slab(p, 2, 6, 8 * 16 * 16 * 4)
        assert ei.value.status == sf.SFSEG_EUNSUPPORTED
    assert lib.sfseg_slab_halo_bytes(None, 0, 0) == -1
    assert lib.sfseg_slab_step(None, None, None, None) == sf.SFSEG_EINVAL


def test_debug_build_exports_the_same_entry_points():
    """The bounds-checked build (libsfseg_debug.so) is built beside the library
    and exports every entry point of include/sfseg.h; it says which it is."""
    import ctypes
    import os
    path = os.path.join(os.path.dirname(sf.LIB_PATH), "libsfseg_debug.so")
    L = ctypes.CDLL(path)
    for name in sf.EXPORTS:
        assert hasattr(L, name), name
    L.sfseg_debug_build.restype = ctypes.c_int32
    assert L.sfseg_debug_build() == 1
    assert sf.load_library().sfseg_debug_build() == (1 if os.environ.get("SFSEG_LIBRARY") == "debug" else 0)


def test_binding_constants_match_the_header():
    """The flag bits, step paths and status codes the binding uses are the
    values include/sfseg.h declares (parsed from the header's enums)."""
    txt = open(os.path.join(ROOT, "include", "sfseg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    declared = {k: int(v) for k, v in re.findall(r"\b(SFSEG_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    checked = 0
    for name, value in declared.items():
        if hasattr(sf, name):
            assert getattr(sf, name) == value, name
            checked += 1
    for name in ("SFSEG_FUSED", "SFSEG_AUTOTUNE", "SFSEG_CLUSTER", "SFSEG_PATH_FAST", "SFSEG_PATH_GENERIC",
                 "SFSEG_PATH_FUSED", "SFSEG_PATH_CLUSTER", "SFSEG_EUNSUPPORTED", "SFSEG_ETIMEOUT"):
        assert name in declared and hasattr(sf, name), name
    assert checked >= 15
    assert set(sf.PATH_NAMES) == {v for k, v in declared.items() if k.startswith("SFSEG_PATH_")}
