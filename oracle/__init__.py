"""FP64 CPU oracle for the SVDLUT transform -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product (the CUDA library and
its Python binding) never calls it, and it shares no code with it.

``svdlut_oracle.c`` holds the arithmetic (Eq. 9 reconstruction, Supp.
Eqs. 12-22 transform and slicing, and their adjoint); this module compiles
it with gcc and marshals numpy arrays.  ``generator.py`` holds the FP64
oracle of the learned factor generator (Supp. Tables 8-12), ``cie94.py`` the
colour-difference term of the training loss (Eq. 11).

Parity status: forward and adjoint are pinned (tests/test_oracle_*.py);
the generator's numeric outputs are "parity unpinned" beyond the paper's
parameter count and finite differences: the paper prints no values.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svdlut_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

PARAM_NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math, OpenMP).  Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i = ctypes.c_int
            lib.oracle_forward.argtypes = [ip, i, i, i] + [dp] * 10 + [i]
            lib.oracle_forward_separable.argtypes = [ip, i, i, i] + [dp] * 10
            lib.oracle_forward_original.argtypes = [ip, i, i, i] + [dp] * 11 + [i]
            lib.oracle_lut3d_apply.argtypes = [i, i, i, i, dp, dp, dp]
            lib.oracle_lut3d_fit2d.argtypes = [i, dp, dp, dp, dp]
            lib.oracle_lut3d_fit2d.restype = ctypes.c_double
            lib.oracle_backward.argtypes = [ip, i, i, i] + [dp] * 19
            lib.oracle_lut_from_svd.argtypes = [i, i, dp, dp, dp, dp]
            lib.oracle_quantize_u8.argtypes = [dp, ctypes.c_void_p, ctypes.c_size_t]
            lib.oracle_u8_to_unit.argtypes = [ctypes.c_void_p, dp, ctypes.c_size_t]
            lib.oracle_u16_to_unit.argtypes = [ctypes.c_void_p, dp, ctypes.c_size_t]
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(d):
    t = d.as_tuple() if hasattr(d, "as_tuple") else tuple(d)
    return (ctypes.c_int * 6)(*t)


def _batched(params, x):
    """Accept unbatched ([3][H][W] + per-image params) or batched inputs."""
    x = _d(x)
    if x.ndim == 3:
        x = x[None]
        params = {k: _d(params[k])[None] for k in PARAM_NAMES}
    else:
        params = {k: _d(params[k]) for k in PARAM_NAMES}
    return params, x


def lut_from_svd(U, S, V):
    """Eq. 9 for one table: U [D][R], S [R], V [D][R] -> T [D][D]."""
    U, S, V = _d(U), _d(S), _d(V)
    D, R = U.shape
    T = np.empty((D, D))
    _load().oracle_lut_from_svd(D, R, _ptr(U), _ptr(S), _ptr(V), _ptr(T))
    return T


def forward(dims, params, x, nthreads: int = 0, separable: bool = False):
    """Y = transform(x) in FP64.  x: [3][H][W] or [B][3][H][W] in [0,1] scale."""
    squeeze = np.asarray(x).ndim == 3
    p, xb = _batched(params, x)
    B, _, H, W = xb.shape
    y = np.empty_like(xb)
    args = [_ptr(p[k]) for k in PARAM_NAMES]
    lib = _load()
    if separable:
        lib.oracle_forward_separable(_dims(dims), B, H, W, *args, _ptr(xb), _ptr(y))
    else:
        lib.oracle_forward(_dims(dims), B, H, W, *args, _ptr(xb), _ptr(y), int(nthreads))
    return y[0] if squeeze else y


def forward_original(dims, params, fusion, x, nthreads: int = 0):
    """The paper's original structure in FP64 (Eqs. 7, 8, 5): K spatial maps,
    the (K+3)->3 1x1 fusion conv, then the 2D LUT transform of the fused
    image.  fusion: [3 (K+3) + 3] or [B][3 (K+3) + 3] (weights [3][K+3], then
    biases [3])."""
    squeeze = np.asarray(x).ndim == 3
    p, xb = _batched(params, x)
    B, _, H, W = xb.shape
    f = _d(fusion)
    if f.ndim == 1:
        f = np.ascontiguousarray(np.broadcast_to(f, (B, f.shape[0])))
    y = np.empty_like(xb)
    _load().oracle_forward_original(_dims(dims), B, H, W, *[_ptr(p[k]) for k in PARAM_NAMES], _ptr(f),
                                    _ptr(xb), _ptr(y), int(nthreads))
    return y[0] if squeeze else y


def lut3d_apply(lut3d, x):
    """Trilinear 3D LUT transform (Eq. 3) in FP64.  lut3d: [3][D][D][D] or
    [B][3][D][D][D] (axes r, g, b per output channel); x: [3][H][W] or
    [B][3][H][W]."""
    squeeze = np.asarray(x).ndim == 3
    xb = _d(x)
    t = _d(lut3d)
    if xb.ndim == 3:
        xb = xb[None]
    if t.ndim == 4:
        t = np.ascontiguousarray(np.broadcast_to(t, (xb.shape[0],) + t.shape))
    B, _, H, W = xb.shape
    y = np.empty_like(xb)
    _load().oracle_lut3d_apply(t.shape[-1], B, H, W, _ptr(t), _ptr(xb), _ptr(y))
    return y[0] if squeeze else y


def lut3d_fit2d(t):
    """Best least-squares fit of one [D][D][D] table by A[i][j] + B[i][k] +
    C[j][k] (second-order ANOVA projection); returns (A, B, C, rms residual)."""
    t = _d(t)
    D = t.shape[0]
    A, Bt, C = np.empty((D, D)), np.empty((D, D)), np.empty((D, D))
    rms = _load().oracle_lut3d_fit2d(D, _ptr(t), _ptr(A), _ptr(Bt), _ptr(C))
    return A, Bt, C, rms


def backward(dims, params, x, dy):
    """Adjoint in FP64: returns dict with dx and d<param> for every parameter."""
    squeeze = np.asarray(x).ndim == 3
    p, xb = _batched(params, x)
    dyb = _d(dy)
    if dyb.ndim == 3:
        dyb = dyb[None]
    B, _, H, W = xb.shape
    out = {"dx": np.empty_like(xb)}
    for k in PARAM_NAMES:
        out["d" + k] = np.empty_like(p[k])
    _load().oracle_backward(_dims(dims), B, H, W, *[_ptr(p[k]) for k in PARAM_NAMES],
                            _ptr(xb), _ptr(dyb), _ptr(out["dx"]),
                            *[_ptr(out["d" + k]) for k in PARAM_NAMES])
    if squeeze:
        out = {k: v[0] for k, v in out.items()}
    return out


def u8_to_unit(v):
    v = np.ascontiguousarray(v, dtype=np.uint8)
    out = np.empty(v.shape, dtype=np.float64)
    _load().oracle_u8_to_unit(v.ctypes.data, _ptr(out), v.size)
    return out


def u16_to_unit(v):
    v = np.ascontiguousarray(v, dtype=np.uint16)
    out = np.empty(v.shape, dtype=np.float64)
    _load().oracle_u16_to_unit(v.ctypes.data, _ptr(out), v.size)
    return out


# Pixel formats of the I/O variants: planar [..][3][H][W] ("f32", "u8",
# "u16") or interleaved [..][H][W][3] ("u8_hwc", "u16_hwc").
PIXEL_FORMATS = ("f32", "u8", "u16", "u8_hwc", "u16_hwc")


def decode(v, fmt):
    """Pixels of format fmt -> planar FP64 in [0,1]: 8-bit codes v/255,
    16-bit codes v/65535 (the 16-bit inputs of Sec. 4.1), float as is."""
    if fmt not in PIXEL_FORMATS:
        raise ValueError(fmt)
    if fmt == "f32":
        return _d(v)
    x = u8_to_unit(v) if fmt.startswith("u8") else u16_to_unit(v)
    if fmt.endswith("_hwc"):
        x = np.moveaxis(x, -1, -3)
    return np.ascontiguousarray(x)


def encode(y, fmt):
    """Planar FP64 result -> format fmt ("f32": as is; 8-bit: quantize_u8)."""
    if fmt == "f32":
        return _d(y)
    if fmt not in ("u8", "u8_hwc"):
        raise ValueError(f"no output encoding {fmt}")
    q = quantize_u8(y)
    return np.ascontiguousarray(np.moveaxis(q, -3, -1)) if fmt == "u8_hwc" else q


def forward_io(dims, params, v, in_fmt, out_fmt, nthreads: int = 0):
    """The forward (Eq. 10) between pixel formats: decode, transform, encode."""
    return encode(forward(dims, params, decode(v, in_fmt), nthreads=nthreads), out_fmt)


def quantize_u8(y):
    y = _d(y)
    out = np.empty(y.shape, dtype=np.uint8)
    _load().oracle_quantize_u8(_ptr(y), out.ctypes.data, y.size)
    return out
