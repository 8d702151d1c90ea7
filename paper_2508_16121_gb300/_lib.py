"""ctypes view of include/svdlut.h.  Argument marshalling only: every step of
the transform runs in libsvdlut.so's CUDA kernels.  Loading fails loudly when
the library has not been built (there is no CPU fallback)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "WORKSPACE", 5: "TIMEOUT"}
F32, U8 = 0, 1

c_int, c_size_t, c_void_p, c_float_p = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p


class Dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("D_t", "rank", "K", "Dsx", "Dsy", "Dsc")]


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")]


class Grads(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("dU", "dS", "dV", "dlut_w", "dg_xy", "dg_xc", "dg_yc", "dgrid_w")]


class Image(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("dims", Dims), ("params", Params),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class LaunchCfg(ctypes.Structure):
    _fields_ = [("block_px", ctypes.c_int32), ("ctas", ctypes.c_int32), ("schedule", ctypes.c_int32)]


SCHED_QUEUE, SCHED_RANGES = 0, 1


class SvdlutError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"svdlut: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsvdlut.so.  Raises if it is missing (no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("SVDLUT_LIB") or _build.LIB
        if build_if_missing and (not os.path.exists(path) or _build.needs_build()):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(
                f"libsvdlut.so is not built ({path}); run paper_2508_16121_gb300.build.build() "
                "-- the CUDA library is required, there is no CPU fallback")
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
        return lib


def _declare(lib):
    P = ctypes.POINTER
    lib.svdlut_last_error.restype = ctypes.c_char_p
    lib.svdlut_version.restype = ctypes.c_char_p
    lib.svdlut_apply.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                 c_void_p]
    lib.svdlut_apply.restype = c_int
    lib.svdlut_backward.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                    P(Grads), c_void_p, c_size_t, c_void_p]
    lib.svdlut_backward.restype = c_int
    lib.svdlut_backward_workspace_size.argtypes = [P(Dims), c_int, c_int, c_int]
    lib.svdlut_backward_workspace_size.restype = c_size_t
    lib.svdlut_apply_batched.argtypes = [P(Image), c_int, c_int, P(LaunchCfg), c_void_p, c_size_t, c_void_p]
    lib.svdlut_apply_batched.restype = c_int
    lib.svdlut_batched_workspace_size.argtypes = [c_int]
    lib.svdlut_batched_workspace_size.restype = c_size_t
    lib.svdlut_batched_tables_workspace_size.argtypes = [P(Image), c_int]
    lib.svdlut_batched_tables_workspace_size.restype = c_size_t
    lib.svdlut_autotune_batched.argtypes = [P(Image), c_int, c_int, c_void_p, c_size_t, c_void_p, c_int,
                                            P(LaunchCfg), ctypes.POINTER(ctypes.c_float)]
    lib.svdlut_autotune_batched.restype = c_int
    lib.svdlut_generator_param_count.argtypes = [c_int]
    lib.svdlut_generator_param_count.restype = c_size_t
    lib.svdlut_generator_workspace_size.argtypes = [c_int, c_int]
    lib.svdlut_generator_workspace_size.restype = c_size_t
    lib.svdlut_generator_forward.argtypes = [c_int, c_void_p, c_int, c_int, c_int, c_void_p, P(Params), c_int,
                                             ctypes.c_uint64, c_void_p, c_size_t, c_void_p]
    lib.svdlut_generator_forward.restype = c_int
    lib.svdlut_generator_backward.argtypes = [c_int, c_void_p, c_int, P(Params), c_void_p, c_int, ctypes.c_uint64,
                                              c_void_p, c_size_t, c_void_p]
    lib.svdlut_generator_backward.restype = c_int
    lib.svdlut_generator_adam.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, c_int, c_void_p]
    lib.svdlut_generator_adam.restype = c_int
    lib.svdlut_mse.argtypes = [c_void_p, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    lib.svdlut_mse.restype = c_int
    lib.svdlut_backward_noalloc.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_void_p, c_void_p,
                                            c_void_p, P(Grads), c_void_p]
    lib.svdlut_backward_noalloc.restype = c_int
    lib.svdlut_apply_original.argtypes = [P(Dims), P(Params), c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                          c_void_p, c_size_t, c_void_p]
    lib.svdlut_apply_original.restype = c_int
    lib.svdlut_apply_original_workspace_size.argtypes = [P(Dims), c_int, c_int, c_int]
    lib.svdlut_apply_original_workspace_size.restype = c_size_t
    lib.svdlut_check_report.argtypes = [c_void_p]
    lib.svdlut_check_report.restype = c_int
    lib.svdlut_apply_cfg.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                     P(LaunchCfg), c_void_p]
    lib.svdlut_apply_cfg.restype = c_int
    lib.svdlut_apply_ws.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                    P(LaunchCfg), c_void_p, c_size_t, c_void_p]
    lib.svdlut_apply_ws.restype = c_int
    lib.svdlut_tensor_core_timeouts.argtypes = [c_void_p]
    lib.svdlut_tensor_core_timeouts.restype = c_int
    lib.svdlut_apply_workspace_size.argtypes = [P(Dims), c_int]
    lib.svdlut_apply_workspace_size.restype = c_size_t
    lib.svdlut_apply_host.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                      c_size_t, c_void_p]
    lib.svdlut_apply_host.restype = c_int
    lib.svdlut_apply_host_workspace_size.argtypes = [c_int, c_int, c_int, c_int]
    lib.svdlut_apply_host_workspace_size.restype = c_size_t
    lib.svdlut_cie94.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, ctypes.c_float, c_void_p, c_int, c_void_p,
                                 c_void_p, c_size_t, c_void_p]
    lib.svdlut_cie94.restype = c_int
    lib.svdlut_apply_io.argtypes = [P(Dims), P(Params), c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p,
                                    c_void_p]
    lib.svdlut_apply_io.restype = c_int
    lib.svdlut_lut3d_apply.argtypes = [c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_size_t,
                                       c_void_p]
    lib.svdlut_lut3d_apply.restype = c_int
    lib.svdlut_lut3d_workspace_size.argtypes = [c_int, c_int]
    lib.svdlut_lut3d_workspace_size.restype = c_size_t
    lib.svdlut_lut3d_fit2d.argtypes = [c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.svdlut_lut3d_fit2d.restype = c_int
    for name, argtypes in _EXTRA.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = argtypes[0]
            f.restype = argtypes[1]


_EXTRA: dict = {}


def check(status: int):
    if status != OK:
        raise SvdlutError(status, load().svdlut_last_error().decode())


# names every build of the library exports (declared in include/svdlut.h)
EXPORTED = ["svdlut_apply", "svdlut_apply_batched", "svdlut_batched_workspace_size", "svdlut_autotune_batched",
            "svdlut_generator_param_count", "svdlut_generator_workspace_size", "svdlut_generator_forward",
            "svdlut_generator_backward", "svdlut_generator_adam", "svdlut_mse", "svdlut_backward", "svdlut_backward_workspace_size", "svdlut_backward_noalloc",
            "svdlut_apply_cfg", "svdlut_apply_original", "svdlut_apply_original_workspace_size", "svdlut_check_report", "svdlut_apply_host", "svdlut_apply_host_workspace_size",
            "svdlut_apply_io", "svdlut_cie94", "svdlut_lut3d_apply", "svdlut_lut3d_workspace_size", "svdlut_lut3d_fit2d", "svdlut_last_error", "svdlut_version"]
