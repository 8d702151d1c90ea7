"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/svdlut.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

import paper_2508_16121_gb300 as svdlut
from paper_2508_16121_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(svdlut_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "svdlut_apply" in names and "svdlut_last_error" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version(lib):
    assert b"sm_103a" in lib.svdlut_version()


def _call_apply(lib, dims, B=1, H=4, W=4, dtype=0, x=0x1000, y=0x100000, params=True):
    p = _lib.Params(U=0x2000, S=0x3000, V=0x4000, lut_w=0x5000, g_xy=0x6000, g_xc=0x7000,
                    g_yc=0x8000, grid_w=0x9000) if params else None
    return lib.svdlut_apply(ctypes.byref(dims) if dims is not None else None,
                            ctypes.byref(p) if p is not None else None, B, H, W, dtype,
                            ctypes.c_void_p(x), ctypes.c_void_p(y), None)


@pytest.mark.parametrize("dims,why", [
    (_lib.Dims(1, 1, 0, 2, 2, 2), "D_t"),
    (_lib.Dims(33, 34, 0, 2, 2, 2), "rank"),
    (_lib.Dims(33, 0, 0, 2, 2, 2), "rank"),
    (_lib.Dims(33, 8, -1, 2, 2, 2), "K"),
    (_lib.Dims(33, 8, 6, 1, 17, 17), "grid"),
])
def test_rejects_bad_dims(lib, dims, why):
    assert _call_apply(lib, dims) == _lib.ERR_INVALID_ARG
    assert why.encode() in lib.svdlut_last_error() or b"grid" in lib.svdlut_last_error()


def test_rejects_unsupported_dims(lib):
    assert _call_apply(lib, _lib.Dims(65, 8, 6, 17, 17, 17)) == _lib.ERR_UNSUPPORTED
    assert _call_apply(lib, _lib.Dims(33, 8, 6, 17, 17, 65)) == _lib.ERR_UNSUPPORTED


def test_rejects_bad_sizes_and_pointers(lib):
    d = _lib.Dims(33, 8, 6, 17, 17, 17)
    assert _call_apply(lib, None) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, params=False) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, H=0) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, B=0) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, dtype=7) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, x=0) == _lib.ERR_INVALID_ARG
    assert _call_apply(lib, d, x=0x1002) == _lib.ERR_INVALID_ARG      # misaligned float
    assert _call_apply(lib, d, x=0x1000, y=0x1010) == _lib.ERR_INVALID_ARG  # overlap
    assert b"overlap" in lib.svdlut_last_error()


def test_missing_grids_rejected_when_k_positive(lib):
    d = _lib.Dims(33, 8, 6, 17, 17, 17)
    p = _lib.Params(U=0x2000, S=0x3000, V=0x4000, lut_w=0x5000)
    st = lib.svdlut_apply(ctypes.byref(d), ctypes.byref(p), 1, 4, 4, 0, ctypes.c_void_p(0x1000),
                          ctypes.c_void_p(0x100000), None)
    assert st == _lib.ERR_INVALID_ARG


def test_dims_inference_from_shapes():
    import numpy as np
    import svdlut_inputs as si
    d = si.spatial_dims(40, 56)
    p = si.make_params(np.random.default_rng(0), d)
    got = svdlut.dims_of({k: np.asarray(v) for k, v in p.items()})
    assert (got.D_t, got.rank, got.K, got.Dsx, got.Dsy, got.Dsc) == d.as_tuple()


def test_check_report_is_unsupported_in_the_normal_build(lib):
    import ctypes
    out = (ctypes.c_uint32 * 4)(7, 7, 7, 7)
    assert lib.svdlut_check_report(out) == 2  # SVDLUT_ERR_UNSUPPORTED
    assert list(out) == [0, 0, 0, 0]
