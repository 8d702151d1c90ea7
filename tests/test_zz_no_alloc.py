"""svdlut_backward_noalloc: the adjoint for callers that cannot allocate
device memory (it uses a fixed scratch array inside the library instead of a
caller workspace).  Checked through the C ABI against svdlut_backward with a
caller workspace, on two calls in a row, within the adjoint tests' tolerance.
This file is collected last on purpose; it also passes run alone."""
import ctypes

import numpy as np
import pytest

import svdlut_inputs as si

pytestmark = pytest.mark.gpu

NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")


def _call(use_noalloc, x, p, dy):
    import torch
    import paper_2508_16121_gb300 as sv
    from paper_2508_16121_gb300 import _lib
    lib = _lib.load(build_if_missing=True)
    xt, gt = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    pt = sv.to_device(p)
    B, _, H, W = x.shape
    d = sv.dims_of(pt)
    ps = sv._param_struct(pt, B, d)
    outs = {"d" + n: torch.full_like(pt[n], float("nan")) for n in NAMES}
    g = _lib.Grads(**{k: (v.data_ptr() if v.numel() else None) for k, v in outs.items()})
    dx = torch.full_like(xt, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if use_noalloc:
        st = lib.svdlut_backward_noalloc(ctypes.byref(d), ctypes.byref(ps), B, H, W, ctypes.c_void_p(xt.data_ptr()),
                                         ctypes.c_void_p(gt.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                                         ctypes.byref(g), stream)
    else:
        need = lib.svdlut_backward_workspace_size(ctypes.byref(d), B, H, W)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        st = lib.svdlut_backward(ctypes.byref(d), ctypes.byref(ps), B, H, W, ctypes.c_void_p(xt.data_ptr()),
                                 ctypes.c_void_p(gt.data_ptr()), ctypes.c_void_p(dx.data_ptr()), ctypes.byref(g),
                                 ctypes.c_void_p(ws.data_ptr()), need, stream)
    assert st == 0, lib.svdlut_last_error()
    torch.cuda.synchronize()
    outs["dx"] = dx
    return {k: v.cpu().numpy().astype(np.float64) for k, v in outs.items()}


def _close(a, r):
    for k in r:
        if r[k].size == 0:
            continue
        assert np.all(np.isfinite(a[k])), k
        assert np.linalg.norm(a[k] - r[k]) <= 1e-4 * max(np.linalg.norm(r[k]), 1e-30) + 1e-6, k
        assert np.abs(a[k] - r[k]).max() <= 1e-3 * np.abs(r[k]).max() + 1e-6, k


def test_noalloc_matches_workspace_path_on_two_calls():
    # two different problems back to back through the shared scratch array
    for seed, (H, W) in ((400, (96, 200)), (401, (64, 128))):
        d = si.spatial_dims(H, W)
        x, p = si.make_batch(seed, 2, H, W, d)
        dy = si.make_upstream(seed + 1, x.shape)
        ref = _call(False, x, p, dy)
        got = _call(True, x, p, dy)
        _close(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2508_16121_gb300 as sv
    from paper_2508_16121_gb300 import _lib
    lib = _lib.load(build_if_missing=True)
    d = si.spatial_dims(2160, 3840)
    p = sv.to_device(si.make_params(np.random.default_rng(402), d))
    dims = sv.dims_of(p)
    B = 16  # 16 x 4K needs far more than the fixed scratch
    pb = {k: v.unsqueeze(0).expand(B, *v.shape).contiguous() for k, v in p.items()}
    ps = sv._param_struct(pb, B, dims)
    dU = torch.empty_like(pb["U"])
    g = _lib.Grads(dU=dU.data_ptr())
    fake = ctypes.c_void_p(0x10000)  # never touched: the size check fails first
    st = lib.svdlut_backward_noalloc(ctypes.byref(dims), ctypes.byref(ps), B, 2160, 3840, fake, fake, None,
                                     ctypes.byref(g), None)
    assert st == _lib.ERR_UNSUPPORTED
    assert b"scratch" in lib.svdlut_last_error()


def test_noalloc_scratch_holds_the_sizes_the_header_names():
    """The header says 8 x 1920x1080 and one 3840x2160 image (D_t=33, rank 8,
    K=8 grids at 1/8 resolution) fit the fixed scratch on a GB300; the
    workspace plan depends on the SM count, so check it on this GPU."""
    import torch
    import paper_2508_16121_gb300 as sv
    from paper_2508_16121_gb300 import _lib
    lib = _lib.load(build_if_missing=True)
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the sizes are stated for a 152-SM GB300")
    for B, H, W in ((8, 1080, 1920), (1, 2160, 3840)):
        d = sv.dims_of(sv.to_device(si.make_params(np.random.default_rng(403), si.spatial_dims(H, W))))
        need = lib.svdlut_backward_workspace_size(ctypes.byref(d), B, H, W)
        assert 0 < need <= 32 << 20, (B, H, W, need)
