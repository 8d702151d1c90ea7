"""GB300-native SVDLUT: fused 2D-LUT transform + 2D bilateral-grid slicing
(arXiv 2508.16121) as hand-written sm_103a CUDA behind a C ABI
(include/svdlut.h).  This module only marshals torch tensors into that ABI;
torch provides device memory and streams.

    import paper_2508_16121_gb300 as svdlut
    y = svdlut.apply(x, params)          # x: [B,3,H,W] or [3,H,W], float32 or uint8, CUDA
    y8 = svdlut.apply_io(x16, params, "u16", "u8")   # 16-bit photo -> 8-bit result
    g = svdlut.backward(x, params, dy)   # adjoint: dx and every parameter gradient
    ys = svdlut.Batch(xs, params_list).run()         # ragged batch, one launch
    p = svdlut.Generator(K, weights).forward(x)      # learned factors for apply

Also: apply_host (host frames), apply_original (the unfused structure),
lut3d_apply / lut3d_fit2d (the 3D LUT and its 2D fit), mse and cie94 (loss
terms), and train.Trainer (end-to-end training of the generator).
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import SvdlutError  # noqa: F401

PARAM_NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")


def _torch():
    import torch
    return torch


def dims_of(params) -> _lib.Dims:
    """Infer (D_t, rank, K, Dsx, Dsy, Dsc) from parameter tensor shapes
    (per-image [3,3,D,R] or batched [B,3,3,D,R] U)."""
    U, gxy, gxc = params["U"], params["g_xy"], params["g_xc"]
    D, R = U.shape[-2], U.shape[-1]
    K, Dsy, Dsx = gxy.shape[-3], gxy.shape[-2], gxy.shape[-1]
    Dsc = gxc.shape[-1]
    return _lib.Dims(D, R, K, Dsx, Dsy, Dsc)


def _param_struct(params, B, d):
    torch = _torch()
    shapes = {"U": (3, 3, d.D_t, d.rank), "S": (3, 3, d.rank), "V": (3, 3, d.D_t, d.rank),
              "lut_w": (3, 4), "g_xy": (d.K, d.Dsy, d.Dsx), "g_xc": (d.K, d.Dsx, d.Dsc),
              "g_yc": (d.K, d.Dsy, d.Dsc), "grid_w": (d.K, 4)}
    ptrs = {}
    for n in PARAM_NAMES:
        t = params[n]
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"param {n} must be a contiguous float32 CUDA tensor")
        want = shapes[n]
        if tuple(t.shape[-len(want):]) != want or t.numel() != B * _numel(want):
            raise ValueError(f"param {n}: shape {tuple(t.shape)} does not match {want} x B={B}")
        ptrs[n] = t.data_ptr() if t.numel() else None
    return _lib.Params(**ptrs)


def _numel(s):
    n = 1
    for v in s:
        n *= v
    return n


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def apply(x, params, out=None, stream=None, ctas=None, workspace=True):
    """Fused SVDLUT apply (Eq. 10).  x: CUDA tensor [B,3,H,W] or [3,H,W],
    float32 or uint8, contiguous.  params: dict of float32 CUDA tensors with
    an optional leading batch axis (see include/svdlut.h).  Returns y with
    x's shape and dtype.  ctas: persistent CTAs to use (default one per SM).
    workspace: True (default) runs svdlut_apply_ws, whose per-image tables
    are precomputed once into a workspace taken from PyTorch's allocator on
    the call's stream; a uint8 CUDA tensor of svdlut_apply_workspace_size
    bytes is used as given; False runs svdlut_apply / svdlut_apply_cfg
    (every CTA rebuilds the tables itself)."""
    torch = _torch()
    squeeze = x.dim() == 3
    xb = x.unsqueeze(0) if squeeze else x
    if xb.dim() != 4 or xb.shape[1] != 3:
        raise ValueError("x must be [B,3,H,W] or [3,H,W]")
    if not xb.is_cuda or not xb.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    if xb.dtype == torch.float32:
        dt = _lib.F32
    elif xb.dtype == torch.uint8:
        dt = _lib.U8
    else:
        raise ValueError("x must be float32 or uint8")
    B, _, H, W = xb.shape
    d = dims_of(params)
    p = _param_struct(params, B, d)
    y = torch.empty_like(xb) if out is None else (out.unsqueeze(0) if squeeze else out)
    if y.shape != xb.shape or y.dtype != xb.dtype or not y.is_contiguous():
        raise ValueError("out must match x in shape and dtype")
    lib = _lib.load()
    if workspace is not False:
        need = lib.svdlut_apply_workspace_size(ctypes.byref(d), B)
        if workspace is True:
            ws = _stream_workspace(torch, need, xb.device, stream)
        else:
            ws = workspace
            if not ws.is_cuda or ws.dtype != torch.uint8 or ws.numel() < need:
                raise ValueError(f"workspace must be a uint8 CUDA tensor of at least {need} bytes")
        cfg = _lib.LaunchCfg(0, int(ctas or 0), 0)
        _lib.check(lib.svdlut_apply_ws(ctypes.byref(d), ctypes.byref(p), B, H, W, dt,
                                       ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.byref(cfg), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       _stream_ptr(stream)))
    elif ctas is None:
        _lib.check(lib.svdlut_apply(ctypes.byref(d), ctypes.byref(p), B, H, W, dt,
                                    ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    _stream_ptr(stream)))
    else:
        cfg = _lib.LaunchCfg(0, int(ctas), 0)
        _lib.check(lib.svdlut_apply_cfg(ctypes.byref(d), ctypes.byref(p), B, H, W, dt,
                                        ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        ctypes.byref(cfg), _stream_ptr(stream)))
    return y[0] if squeeze else y


def _stream_workspace(torch, nbytes, device, stream):
    """Device scratch of nbytes from PyTorch's caching allocator, owned by the
    stream the call runs on (so concurrent streams never share it)."""
    if stream is None:
        return torch.empty(nbytes, dtype=torch.uint8, device=device)
    with torch.cuda.stream(stream):
        return torch.empty(nbytes, dtype=torch.uint8, device=device)


# pixel formats of apply_io (svdlut_pixfmt): code, element dtypes, interleaved?
PIXEL_FORMATS = {"f32": (0, ("float32",), False), "u8": (1, ("uint8",), False),
                 "u16": (2, ("uint16", "int16"), False), "u8_hwc": (3, ("uint8",), True),
                 "u16_hwc": (4, ("uint16", "int16"), True)}


def _pix_tensor(t, fmt, what):
    torch = _torch()
    if fmt not in PIXEL_FORMATS:
        raise ValueError(f"unknown pixel format {fmt!r}")
    _, dts, hwc = PIXEL_FORMATS[fmt]
    single = t.dim() == 3
    tb = t.unsqueeze(0) if single else t
    if tb.dim() != 4 or tb.shape[3 if hwc else 1] != 3:
        raise ValueError(f"{what} must be {'[B,H,W,3]' if hwc else '[B,3,H,W]'} (or without B) for {fmt}")
    if str(tb.dtype).replace("torch.", "") not in dts or not tb.is_cuda or not tb.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor of {' or '.join(dts)} for {fmt}")
    H, W = (tb.shape[1], tb.shape[2]) if hwc else (tb.shape[2], tb.shape[3])
    return tb, single, H, W


def apply_io(x, params, in_format, out_format, out=None, stream=None):
    """The fused transform between pixel formats (svdlut_apply_io): 16-bit
    ("u16", "u16_hwc") and 8-bit inputs are decoded and 8-bit outputs
    encoded inside the kernel.  Formats: "f32", "u8", "u16" planar
    [B,3,H,W]; "u8_hwc", "u16_hwc" interleaved [B,H,W,3].  Supported pairs:
    u16->u8, u16->f32, u8_hwc->u8_hwc, u16_hwc->u8_hwc (and f32->f32,
    u8->u8 as apply)."""
    torch = _torch()
    xb, single, H, W = _pix_tensor(x, in_format, "x")
    B = xb.shape[0]
    hwc_out = PIXEL_FORMATS.get(out_format, (0, (), False))[2]
    if out is None:
        if out_format not in ("f32", "u8", "u8_hwc"):
            raise ValueError(f"no output encoding {out_format!r}")
        dt = torch.float32 if out_format == "f32" else torch.uint8
        out = torch.empty((B, H, W, 3) if hwc_out else (B, 3, H, W), dtype=dt, device=xb.device)
        yb = out
    else:
        yb, _, Ho, Wo = _pix_tensor(out, out_format, "out")
        if (yb.shape[0], Ho, Wo) != (B, H, W):
            raise ValueError("out must hold the same images as x")
    d = dims_of(params)
    p = _param_struct(params, B, d)
    _lib.check(_lib.load().svdlut_apply_io(ctypes.byref(d), ctypes.byref(p), B, H, W, PIXEL_FORMATS[in_format][0],
                                           ctypes.c_void_p(xb.data_ptr()), PIXEL_FORMATS[out_format][0],
                                           ctypes.c_void_p(yb.data_ptr()), _stream_ptr(stream)))
    return yb[0] if single else yb


_host_ws = {}


def apply_host(x, params, out=None, stream=None):
    """Fused apply on host images (svdlut_apply_host): x is a CPU tensor
    [B,3,H,W] or [3,H,W] (float32 or uint8, contiguous), params are CUDA
    tensors as for apply.  Pinned x and out are read and written in place by
    the kernel over the CPU-GPU link; pageable ones go through banded copies
    overlapped with the transform.  The result (a CPU tensor, pinned when
    allocated here) is complete once `stream` (default: the current stream)
    has reached the end of the call."""
    torch = _torch()
    squeeze = x.dim() == 3
    xb = x.unsqueeze(0) if squeeze else x
    if xb.dim() != 4 or xb.shape[1] != 3:
        raise ValueError("x must be [B,3,H,W] or [3,H,W]")
    if xb.is_cuda or not xb.is_contiguous():
        raise ValueError("x must be a contiguous host tensor")
    if xb.dtype == torch.float32:
        dt = _lib.F32
    elif xb.dtype == torch.uint8:
        dt = _lib.U8
    else:
        raise ValueError("x must be float32 or uint8")
    B, _, H, W = xb.shape
    d = dims_of(params)
    p = _param_struct(params, B, d)
    y = torch.empty(xb.shape, dtype=xb.dtype, pin_memory=True) if out is None else (out.unsqueeze(0) if squeeze else out)
    if y.shape != xb.shape or y.dtype != xb.dtype or y.is_cuda or not y.is_contiguous():
        raise ValueError("out must be a host tensor matching x in shape and dtype")
    lib = _lib.load()
    sp = _stream_ptr(stream)
    ws_ptr, ws_bytes = None, 0
    if not (xb.is_pinned() and y.is_pinned()):  # pinned frames are used in place, no workspace
        need = lib.svdlut_apply_host_workspace_size(B, H, W, dt)
        dev = next(iter(params.values())).device
        key = (str(dev), sp.value)  # one workspace per device and stream: calls on one stream are ordered
        ws = _host_ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            _host_ws[key] = ws
        ws_ptr, ws_bytes = ws.data_ptr(), ws.numel()
    _lib.check(lib.svdlut_apply_host(ctypes.byref(d), ctypes.byref(p), B, H, W, dt, ctypes.c_void_p(xb.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(ws_ptr), ws_bytes, sp))
    return y[0] if squeeze else y


def original_workspace_bytes(params, B, H, W):
    """Device workspace of apply_original for B images of H x W."""
    return int(_lib.load().svdlut_apply_original_workspace_size(ctypes.byref(dims_of(params)), B, H, W))


def apply_original(x, params, fusion, out=None, workspace=None, stream=None):
    """The paper's original, unfused structure (svdlut_apply_original): K
    spatial maps and the fused image go through HBM.  x: float32 CUDA tensor
    [B,3,H,W] or [3,H,W]; fusion: CUDA tensor [3 (K+3) + 3] or
    [B, 3 (K+3) + 3] (1x1 conv weights [3][K+3], then biases [3])."""
    torch = _torch()
    squeeze = x.dim() == 3
    xb = x.unsqueeze(0) if squeeze else x
    if xb.dim() != 4 or xb.shape[1] != 3 or xb.dtype != torch.float32 or not xb.is_cuda or not xb.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor [B,3,H,W] or [3,H,W]")
    B, _, H, W = xb.shape
    d = dims_of(params)
    p = _param_struct(params, B, d)
    nf = 3 * (d.K + 3) + 3
    f = fusion.reshape(-1, nf)
    if f.shape[0] == 1 and B > 1:
        f = f.expand(B, nf)
    f = f.to(torch.float32).contiguous()
    if f.shape != (B, nf) or not f.is_cuda:
        raise ValueError(f"fusion must hold {nf} floats per image on the GPU")
    y = torch.empty_like(xb) if out is None else (out.unsqueeze(0) if squeeze else out)
    lib = _lib.load()
    need = lib.svdlut_apply_original_workspace_size(ctypes.byref(d), B, H, W)
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        torch.empty(need, dtype=torch.uint8, device=xb.device)
    _lib.check(lib.svdlut_apply_original(ctypes.byref(d), ctypes.byref(p), ctypes.c_void_p(f.data_ptr()), B, H, W,
                                         ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return y[0] if squeeze else y


def _lut3d_tensor(lut3d):
    torch = _torch()
    t = lut3d.unsqueeze(0) if lut3d.dim() == 4 else lut3d
    if (t.dim() != 5 or t.shape[1] != 3 or not (t.shape[2] == t.shape[3] == t.shape[4])
            or t.dtype != torch.float32 or not t.is_cuda):
        raise ValueError("lut3d must be a float32 CUDA tensor [B,3,D,D,D] or [3,D,D,D]")
    return t.contiguous()


def lut3d_apply(x, lut3d, out=None, workspace=None, stream=None):
    """3D LUT transform (Eq. 3, svdlut_lut3d_apply): trilinear lookup of
    lut3d [B,3,D,D,D] (or [3,D,D,D] shared by the batch), index [r][g][b],
    at every pixel of x (float32 CUDA [B,3,H,W] or [3,H,W])."""
    torch = _torch()
    squeeze = x.dim() == 3
    xb = x.unsqueeze(0) if squeeze else x
    if xb.dim() != 4 or xb.shape[1] != 3 or xb.dtype != torch.float32 or not xb.is_cuda or not xb.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor [B,3,H,W] or [3,H,W]")
    B, _, H, W = xb.shape
    t = _lut3d_tensor(lut3d)
    if t.shape[0] == 1 and B > 1:
        t = t.expand(B, *t.shape[1:]).contiguous()
    if t.shape[0] != B:
        raise ValueError(f"lut3d holds {t.shape[0]} tables for {B} images")
    D = t.shape[-1]
    y = torch.empty_like(xb) if out is None else (out.unsqueeze(0) if squeeze else out)
    lib = _lib.load()
    need = lib.svdlut_lut3d_workspace_size(D, B)
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        torch.empty(need, dtype=torch.uint8, device=xb.device)
    _lib.check(lib.svdlut_lut3d_apply(D, ctypes.c_void_p(t.data_ptr()), B, H, W, ctypes.c_void_p(xb.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      _stream_ptr(stream)))
    return y[0] if squeeze else y


def lut3d_fit2d(lut3d, stream=None):
    """Least-squares fit of each 3D table by A[r][g] + Bt[r][b] + C[g][b]
    (the hypothesis of Eq. 4; svdlut_lut3d_fit2d).  Returns (tables
    [B,3,3,D,D] in pair order (A, Bt, C), rms [B,3])."""
    torch = _torch()
    t = _lut3d_tensor(lut3d)
    B, D = t.shape[0], t.shape[-1]
    tables = torch.empty(B, 3, 3, D, D, dtype=torch.float32, device=t.device)
    rms = torch.empty(B, 3, dtype=torch.float32, device=t.device)
    _lib.check(_lib.load().svdlut_lut3d_fit2d(D, ctypes.c_void_p(t.data_ptr()), B, ctypes.c_void_p(tables.data_ptr()),
                                              ctypes.c_void_p(rms.data_ptr()), _stream_ptr(stream)))
    return tables, rms


def fit_params(tables):
    """svdlut parameters that run 2D tables [B,3,3,D,D] (e.g. from
    lut3d_fit2d) through apply at full rank: U = the tables, S = 1, V = I,
    lut_w = (1, 1, 1, 0), no grids."""
    torch = _torch()
    B, D = tables.shape[0], tables.shape[-1]
    dev = tables.device
    V = torch.eye(D, dtype=torch.float32, device=dev).expand(B, 3, 3, D, D).contiguous()
    lut_w = torch.tensor([1.0, 1.0, 1.0, 0.0], device=dev).expand(B, 3, 4).contiguous()
    none = torch.empty(B, 0, 2, 2, device=dev)
    return dict(U=tables.contiguous(), S=torch.ones(B, 3, 3, D, device=dev), V=V, lut_w=lut_w,
                g_xy=none, g_xc=none, g_yc=none, grid_w=torch.empty(B, 0, 4, device=dev))


def check_report():
    """Index-check status of a library built with -DSVDLUT_CHECK_BOUNDS:
    dict(failures, site, index, limit) of the first failure since the last
    call (and clears it); None for the normal build."""
    lib = _lib.load()
    out = (ctypes.c_uint32 * 4)()
    st = lib.svdlut_check_report(out)
    if st == 2:  # SVDLUT_ERR_UNSUPPORTED: normal build
        return None
    _lib.check(st)
    return {"failures": out[0], "site": out[1], "index": out[2], "limit": out[3]}


def to_device(params, device="cuda"):
    """numpy / torch parameter dict -> contiguous float32 tensors on device."""
    torch = _torch()
    return {k: torch.as_tensor(v, dtype=torch.float32).contiguous().to(device) for k, v in params.items()}


def backward(x, params, dy, want=("dx",) + tuple("d" + n for n in PARAM_NAMES), workspace=None, stream=None):
    """Adjoint of apply for float32 images (svdlut_backward).  Returns a dict
    with the requested gradients ('dx', 'dU', 'dS', 'dV', 'dlut_w', 'dg_xy',
    'dg_xc', 'dg_yc', 'dgrid_w'), each shaped like its input.  Deterministic:
    identical inputs give identical bits."""
    torch = _torch()
    squeeze = x.dim() == 3
    xb = x.unsqueeze(0) if squeeze else x
    gb = dy.unsqueeze(0) if squeeze else dy
    if xb.dtype != torch.float32 or gb.dtype != torch.float32:
        raise ValueError("backward needs float32 x and dy")
    if gb.shape != xb.shape or not xb.is_contiguous() or not gb.is_contiguous():
        raise ValueError("dy must be contiguous and shaped like x")
    B, _, H, W = xb.shape
    d = dims_of(params)
    p = _param_struct(params, B, d)
    out = {}
    ptrs = {}
    for n in PARAM_NAMES:
        if "d" + n in want:
            t = torch.empty_like(params[n])
            out["d" + n] = t
            ptrs["d" + n] = t.data_ptr() if t.numel() else None
    g = _lib.Grads(**ptrs)
    dx = torch.empty_like(xb) if "dx" in want else None
    lib = _lib.load()
    need = lib.svdlut_backward_workspace_size(ctypes.byref(d), B, H, W)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=xb.device)
    _lib.check(lib.svdlut_backward(ctypes.byref(d), ctypes.byref(p), B, H, W, ctypes.c_void_p(xb.data_ptr()),
                                   ctypes.c_void_p(gb.data_ptr()),
                                   ctypes.c_void_p(dx.data_ptr()) if dx is not None else None,
                                   ctypes.byref(g), ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                   _stream_ptr(stream)))
    if dx is not None:
        out["dx"] = dx[0] if squeeze else dx
    return out


class _ApplyFn:
    """torch.autograd.Function around svdlut_apply / svdlut_backward."""
    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            torch = _torch()

            class Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, *tensors):
                    params = dict(zip(PARAM_NAMES, tensors))
                    ctx.save_for_backward(x, *tensors)
                    return apply(x, params)

                @staticmethod
                def backward(ctx, gy):
                    x, *tensors = ctx.saved_tensors
                    params = dict(zip(PARAM_NAMES, tensors))
                    want = []
                    if ctx.needs_input_grad[0]:
                        want.append("dx")
                    for i, n in enumerate(PARAM_NAMES):
                        if ctx.needs_input_grad[1 + i]:
                            want.append("d" + n)
                    g = backward(x, params, gy.contiguous(), want=tuple(want))
                    return (g.get("dx"),) + tuple(g.get("d" + n) for n in PARAM_NAMES)

            cls._cls = Fn
        return cls._cls


def apply_autograd(x, params):
    """Differentiable apply (float32): gradients flow to x and every
    parameter tensor through svdlut_backward."""
    return _ApplyFn.get().apply(x, *[params[n] for n in PARAM_NAMES])


class Batch:
    """A ragged batch for svdlut_apply_batched: images of uneven sizes, each
    with its own parameter dict (per-image layouts, no batch axis).  Holds the
    host descriptor array and the device workspace so that repeated calls
    (and CUDA-graph capture of a call) marshal nothing new."""

    def __init__(self, xs, params_list, outs=None, tables=True):
        """tables: give svdlut_apply_batched the workspace for the per-image
        tables (computed once per call instead of in every CTA)."""
        torch = _torch()
        if len(xs) != len(params_list) or not xs:
            raise ValueError("need one parameter dict per image")
        self.dtype = _lib.U8 if xs[0].dtype == torch.uint8 else _lib.F32
        self.xs = list(xs)
        self.params = list(params_list)
        self.outs = list(outs) if outs is not None else [torch.empty_like(x) for x in xs]
        n = len(xs)
        self.imgs = (_lib.Image * n)()
        for i, (x, p, y) in enumerate(zip(self.xs, self.params, self.outs)):
            if x.dim() != 3 or x.shape[0] != 3 or not x.is_contiguous() or not x.is_cuda:
                raise ValueError("each image must be a contiguous [3,H,W] CUDA tensor")
            if (x.dtype == torch.uint8) != (self.dtype == _lib.U8) or y.shape != x.shape or y.dtype != x.dtype:
                raise ValueError("all images (and outputs) must share one dtype and match in shape")
            d = dims_of(p)
            self.imgs[i] = _lib.Image(x.shape[1], x.shape[2], d, _param_struct(p, 1, d),
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
        lib = _lib.load()
        need = lib.svdlut_batched_tables_workspace_size(self.imgs, n) if tables else \
            lib.svdlut_batched_workspace_size(n)
        self.ws = torch.zeros(max(int(need), 4), dtype=torch.uint8, device=xs[0].device)
        self.cfg = None

    def run(self, stream=None):
        lib = _lib.load()
        cfg = ctypes.byref(self.cfg) if self.cfg is not None else None
        _lib.check(lib.svdlut_apply_batched(self.imgs, len(self.xs), self.dtype, cfg,
                                            ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                            _stream_ptr(stream)))
        return self.outs

    def tune_key(self):
        """Key of this batch's launch-shape choice: GPU model, dtype and the
        per-image sizes and transform dims."""
        torch = _torch()
        name = torch.cuda.get_device_name(self.xs[0].device)
        def dims_str(p):
            d = dims_of(p)
            return ",".join(str(getattr(d, n)) for n, _ in _lib.Dims._fields_)
        shapes = ";".join(f"{x.shape[1]}x{x.shape[2]}:{dims_str(p)}" for x, p in zip(self.xs, self.params))
        return f"{name}|{'u8' if self.dtype == _lib.U8 else 'f32'}|{shapes}"

    def autotune(self, reps=5, stream=None, cache=None):
        """Time a set of block sizes and both block schedules on this batch
        (native autotuner) and keep the fastest launch shape (self.cfg);
        returns (block_px, ms).  cache: path of a JSON file of
        earlier choices keyed by tune_key() (default: $SVDLUT_AUTOTUNE_CACHE,
        none if unset); a hit skips the timing and returns (block_px, None)."""
        import json
        import os
        path = cache if cache is not None else os.environ.get("SVDLUT_AUTOTUNE_CACHE")
        key = self.tune_key()
        table = {}
        if path and os.path.exists(path):
            with open(path) as f:
                table = json.load(f)
            if key in table:
                self.cfg = _lib.LaunchCfg(int(table[key]["block_px"]), int(table[key].get("ctas", 0)),
                                          int(table[key].get("schedule", 0)))
                return self.cfg.block_px, None
        lib = _lib.load()
        best = _lib.LaunchCfg()
        ms = ctypes.c_float()
        _lib.check(lib.svdlut_autotune_batched(self.imgs, len(self.xs), self.dtype,
                                               ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                               _stream_ptr(stream), reps, ctypes.byref(best), ctypes.byref(ms)))
        self.cfg = best
        if path:
            table[key] = {"block_px": int(best.block_px), "ctas": int(best.ctas), "schedule": int(best.schedule),
                          "ms": float(ms.value)}
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        return best.block_px, ms.value


def apply_batched(xs, params_list, outs=None, stream=None):
    """One persistent launch over images of uneven sizes (svdlut_apply_batched)."""
    return Batch(xs, params_list, outs).run(stream)


GEN_DT, GEN_RANK, GEN_DS = 33, 8, 17


class Generator:
    """The learned factor generator (svdlut_generator_* in the C ABI).

    weights: FP32 CUDA tensor of svdlut_generator_param_count(K) values (the
    layout documented in include/svdlut.h).  forward() returns the parameter
    dict svdlut.apply consumes (leading batch axis), backward() the weight
    gradient of sum(dparams * params) for the last forward."""

    def __init__(self, K, weights, max_batch=64):
        torch = _torch()
        lib = _lib.load()
        self.K = int(K)
        self.n = int(lib.svdlut_generator_param_count(self.K))
        if weights.numel() != self.n or weights.dtype != torch.float32 or not weights.is_cuda:
            raise ValueError(f"weights must be {self.n} float32 values on the GPU")
        self.weights = weights.contiguous()
        self.max_batch = int(max_batch)
        self.ws = torch.empty(int(lib.svdlut_generator_workspace_size(self.K, self.max_batch)), dtype=torch.uint8,
                              device=weights.device)
        self.last = None

    def dims(self):
        return _lib.Dims(GEN_DT, GEN_RANK, self.K, GEN_DS, GEN_DS, GEN_DS)

    def empty_params(self, B):
        torch = _torch()
        dev = self.weights.device
        K, D, R, S = self.K, GEN_DT, GEN_RANK, GEN_DS
        shapes = {"U": (B, 3, 3, D, R), "S": (B, 3, 3, R), "V": (B, 3, 3, D, R), "lut_w": (B, 3, 4),
                  "g_xy": (B, K, S, S), "g_xc": (B, K, S, S), "g_yc": (B, K, S, S), "grid_w": (B, K, 4)}
        return {k: torch.empty(v, dtype=torch.float32, device=dev) for k, v in shapes.items()}

    @staticmethod
    def _ptrs(d):
        return _lib.Params(**{k: (d[k].data_ptr() if d[k].numel() else None) for k in PARAM_NAMES})

    def forward(self, x, training=False, seed=0, out=None, stream=None):
        B, C, H, W = x.shape
        if C != 3 or B > self.max_batch or x.dtype != _torch().float32 or not x.is_contiguous():
            raise ValueError("x must be a contiguous float32 [B,3,H,W] with B <= max_batch")
        out = out if out is not None else self.empty_params(B)
        lib = _lib.load()
        _lib.check(lib.svdlut_generator_forward(self.K, ctypes.c_void_p(self.weights.data_ptr()), B, H, W,
                                                ctypes.c_void_p(x.data_ptr()), ctypes.byref(self._ptrs(out)),
                                                int(bool(training)), ctypes.c_uint64(seed),
                                                ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                                _stream_ptr(stream)))
        self.last = (B, int(bool(training)), int(seed))
        return out

    def backward(self, dparams, dweights=None, stream=None):
        torch = _torch()
        if self.last is None:
            raise RuntimeError("backward needs a forward first")
        B, training, seed = self.last
        dw = dweights if dweights is not None else torch.empty_like(self.weights)
        lib = _lib.load()
        _lib.check(lib.svdlut_generator_backward(self.K, ctypes.c_void_p(self.weights.data_ptr()), B,
                                                 ctypes.byref(self._ptrs(dparams)), ctypes.c_void_p(dw.data_ptr()),
                                                 training, ctypes.c_uint64(seed),
                                                 ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                                 _stream_ptr(stream)))
        return dw


def adam_step(weights, grads, m, v, step, lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on FP32 CUDA tensors (svdlut_generator_adam)."""
    lib = _lib.load()
    _lib.check(lib.svdlut_generator_adam(ctypes.c_void_p(weights.data_ptr()), ctypes.c_void_p(grads.data_ptr()),
                                         ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), weights.numel(),
                                         lr, beta1, beta2, eps, int(step), _stream_ptr(stream)))


CIE94_WEIGHT = 0.005  # lambda_c of the training loss (Eq. 11)


def cie94(y, target, weight=1.0, dy=None, accumulate=False, ws=None, stream=None):
    """Colour-difference term of the loss (svdlut_cie94): mean CIE94 Delta E
    between y and the reference target, float32 CUDA [B,3,H,W] or [3,H,W]
    sRGB images, as a 0-d CUDA tensor; if dy is given, weight times the
    gradient is written into it (added to it with accumulate=True)."""
    torch = _torch()
    yb = y.unsqueeze(0) if y.dim() == 3 else y
    tb = target.unsqueeze(0) if target.dim() == 3 else target
    for t, what in ((yb, "y"), (tb, "target")):
        if t.dim() != 4 or t.shape[1] != 3 or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous float32 CUDA tensor [B,3,H,W] or [3,H,W]")
    if yb.shape != tb.shape or (dy is not None and (dy.numel() != yb.numel() or not dy.is_contiguous())):
        raise ValueError("y, target and dy must have the same shape")
    B, _, H, W = yb.shape
    loss = torch.empty((), dtype=torch.float32, device=y.device)
    ws = ws if ws is not None else torch.empty(4096, dtype=torch.uint8, device=y.device)
    _lib.check(_lib.load().svdlut_cie94(ctypes.c_void_p(yb.data_ptr()), ctypes.c_void_p(tb.data_ptr()), B, H, W,
                                        float(weight), ctypes.c_void_p(dy.data_ptr()) if dy is not None else None,
                                        int(bool(accumulate)), ctypes.c_void_p(loss.data_ptr()),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return loss


def mse(y, target, dy=None, ws=None, stream=None):
    """MSE loss (0-d CUDA tensor) and, into dy if given, its gradient."""
    torch = _torch()
    loss = torch.empty((), dtype=torch.float32, device=y.device)
    ws = ws if ws is not None else torch.empty(4096, dtype=torch.uint8, device=y.device)
    lib = _lib.load()
    _lib.check(lib.svdlut_mse(ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(target.data_ptr()), y.numel(),
                              ctypes.c_void_p(dy.data_ptr()) if dy is not None else None,
                              ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                              _stream_ptr(stream)))
    return loss
