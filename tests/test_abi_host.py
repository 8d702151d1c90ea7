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


def _params():
    return _lib.Params(U=0x2000, S=0x3000, V=0x4000, lut_w=0x5000, g_xy=0x6000, g_xc=0x7000, g_yc=0x8000,
                       grid_w=0x9000)


def test_apply_io_rejects_bad_formats_and_pointers(lib):
    d, p = _lib.Dims(33, 8, 6, 17, 17, 17), _params()
    call = lambda fi, fo, x=0x10000, y=0x1000000, H=4, W=4: lib.svdlut_apply_io(  # noqa: E731
        ctypes.byref(d), ctypes.byref(p), 1, H, W, fi, ctypes.c_void_p(x), fo, ctypes.c_void_p(y), None)
    assert call(9, 1) == _lib.ERR_INVALID_ARG                     # unknown input format
    assert call(2, 1, x=0) == _lib.ERR_INVALID_ARG                # null input
    assert call(2, 1, x=0x10001) == _lib.ERR_INVALID_ARG          # 16-bit input at an odd address
    assert call(2, 1, x=0x10000, y=0x10004) == _lib.ERR_INVALID_ARG  # overlapping images
    assert call(1, 0) == _lib.ERR_UNSUPPORTED                     # 8-bit in, float out: not built
    assert call(0, 2) == _lib.ERR_UNSUPPORTED                     # 16-bit output: not built
    assert call(2, 1, H=0) == _lib.ERR_INVALID_ARG


def test_lut3d_and_loss_entries_reject_bad_arguments(lib):
    c = ctypes.c_void_p
    assert lib.svdlut_lut3d_apply(34, c(0x1000), 1, 4, 4, c(0x10000), c(0x20000), c(0x30000), 1 << 20,
                                  None) == _lib.ERR_INVALID_ARG          # D > 33
    assert lib.svdlut_lut3d_apply(33, c(0x1000), 1, 4, 4, c(0x10000), c(0x20000), c(0x30000), 16,
                                  None) == _lib.ERR_WORKSPACE            # workspace too small
    assert lib.svdlut_lut3d_workspace_size(33, 2) == 2 * 33 ** 3 * 16
    assert lib.svdlut_lut3d_fit2d(1, c(0x1000), 1, c(0x2000), c(0x3000), None) == _lib.ERR_INVALID_ARG
    assert lib.svdlut_lut3d_fit2d(33, None, 1, c(0x2000), c(0x3000), None) == _lib.ERR_INVALID_ARG
    assert lib.svdlut_cie94(c(0x1000), c(0x2000), 1, 4, 4, 1.0, None, 0, c(0x3000), c(0x4000), 16,
                            None) == _lib.ERR_WORKSPACE
    assert lib.svdlut_cie94(None, c(0x2000), 1, 4, 4, 1.0, None, 0, c(0x3000), c(0x4000), 4096,
                            None) == _lib.ERR_INVALID_ARG
    assert lib.svdlut_cie94(c(0x1002), c(0x2000), 1, 4, 4, 1.0, None, 0, c(0x3000), c(0x4000), 4096,
                            None) == _lib.ERR_INVALID_ARG                # misaligned float array


def test_apply_original_rejects_bad_arguments(lib):
    d, p = _lib.Dims(33, 8, 6, 17, 17, 17), _params()
    c = ctypes.c_void_p
    need = lib.svdlut_apply_original_workspace_size(ctypes.byref(d), 1, 4, 4)
    assert need > 0
    args = lambda x, y, ws, nws: (ctypes.byref(d), ctypes.byref(p), c(0x1000), 1, 4, 4, c(x), c(y), c(ws), nws,  # noqa: E731
                                  None)
    assert lib.svdlut_apply_original(*args(0x10000, 0x10010, 0x100000, need)) == _lib.ERR_INVALID_ARG  # overlap
    assert lib.svdlut_apply_original(*args(0x10000, 0x20000, 0x100000, need - 1)) == _lib.ERR_WORKSPACE
    assert lib.svdlut_apply_original(*args(0x10000, 0x20000, 0x100010, need)) == _lib.ERR_INVALID_ARG  # ws alignment


def test_header_is_plain_c():
    """include/svdlut.h compiles as C99 (no C++ or CUDA types leak into the
    ABI) and as C++."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    hdr = os.path.join(ROOT, "include", "svdlut.h")
    r = subprocess.run([cc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Wextra", "-Werror", hdr],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([cc, "-fsyntax-only", "-x", "c++", "-Wall", "-Werror", hdr], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_generator_workspace_size_holds_the_activations(lib):
    """svdlut_generator_workspace_size (host-only): 0 for invalid K or B,
    whole 256-byte units, growing with the batch, and at least the thumbnail
    and the five convolution activations that the backward pass reads back
    (channels 8/16/32/64/64 at 128..8 pixels square, Supp. A, Table 8)."""
    assert lib.svdlut_generator_workspace_size(-1, 4) == 0
    assert lib.svdlut_generator_workspace_size(8, 0) == 0
    ch, sz = [8, 16, 32, 64, 64], [128, 64, 32, 16, 8]
    prev = 0
    for B in (1, 2, 3, 17, 64):
        n = lib.svdlut_generator_workspace_size(8, B)
        assert n % 256 == 0 and n > prev
        floats = B * 3 * 256 * 256 + sum(B * c * s * s for c, s in zip(ch, sz))
        assert n >= 4 * floats
        prev = n
