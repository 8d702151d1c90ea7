"""GPU parity of svdlut_apply (through the C ABI) against the FP64 oracle.

Bar: max-abs <= 2e-5 on FP32 outputs; <= 1 LSB on 8-bit outputs.  Sizes
span several 128x32 tiles with ragged tails, plus the degenerate shapes
(W = 1, H = 1, 1x1), W not a multiple of 4, misaligned views, clamped
inputs, every K regime, D_t in {2, 17, 33} and the full rank.
"""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def run(sv, x, p, dtype="f32"):
    import torch
    xt = torch.from_numpy(x).cuda()
    y = sv.apply(xt, sv.to_device(p))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def check_f32(sv, d, x, p, tol=TOL):
    y = run(sv, x, p).astype(np.float64)
    ref = oracle.forward(d, p, x)
    err = np.abs(y - ref).max()
    assert err <= tol, err
    return err


@pytest.mark.parametrize("HW", [(256, 256), (1, 1), (1, 37), (29, 1), (33, 130), (67, 257), (130, 515)])
def test_f32_spatial_dims(sv, HW):
    H, W = HW
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(0) + H * 7 + W, 1, H, W, d)
    check_f32(sv, d, x, p)


@pytest.mark.parametrize("d", [si.paper_dims(), si.Dims(2, 1, 3, 2, 2, 2), si.Dims(17, 8, 8, 9, 5, 33),
                               si.Dims(33, 33, 0, 2, 2, 2), si.Dims(5, 3, 1, 3, 4, 2), si.Dims(33, 8, 48, 17, 17, 33),
                               si.Dims(33, 33, 48, 9, 7, 64)])  # the largest sizes the ABI accepts
def test_f32_dims_variants(sv, d):
    x, p = si.make_batch(77, 1, 70, 260, d)
    check_f32(sv, d, x, p)


def test_batch_of_three(sv):
    d = si.spatial_dims(48, 200)
    x, p = si.make_batch(5, 3, 48, 200, d)
    check_f32(sv, d, x, p)


def test_batch_larger_than_one_launch_chunk(sv):
    d = si.Dims(9, 2, 3, 4, 4, 5)
    x, p = si.make_batch(6, 19, 9, 20, d)
    check_f32(sv, d, x, p)


def test_batches_of_64_image_launches_equal_16_image_launches(sv):
    """Batches above 16 images are launched 64 at a time (70 images: two
    launches); each image's result equals the oracle and, bit for bit, the
    same image transformed in a batch of at most 16 (the 16-image launch)."""
    d = si.spatial_dims(12, 40)
    x, p = si.make_batch(12, 70, 12, 40, d)
    y = run(sv, x, p)
    assert np.abs(y.astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL
    for b0, b1 in ((0, 16), (60, 70)):
        part = {k: v[b0:b1] for k, v in p.items()}
        assert np.array_equal(run(sv, np.ascontiguousarray(x[b0:b1]), part), y[b0:b1])


def test_identity_reproduces_input(sv):
    d = si.spatial_dims(40, 300)
    x = si.make_image(np.random.default_rng(3), 40, 300)
    p = {k: v.astype(np.float32) for k, v in si.identity_params(d).items()}
    y = run(sv, x, p)
    assert np.abs(y - x).max() <= 1e-6


def test_clamped_inputs(sv):
    d = si.spatial_dims(20, 44)
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.5, 1.5, size=(3, 20, 44)).astype(np.float32)
    p = si.make_params(rng, d)
    check_f32(sv, d, x, p)


def test_misaligned_views_use_scalar_path(sv):
    import torch
    d = si.spatial_dims(16, 64)
    x, p = si.make_batch(8, 1, 16, 64, d)
    buf = torch.zeros(x.size + 1, dtype=torch.float32, device="cuda")
    xv = buf[1:].view(x.shape)
    xv.copy_(torch.from_numpy(x))
    out = torch.zeros(x.size + 1, dtype=torch.float32, device="cuda")
    yv = out[1:].view(x.shape)
    sv.apply(xv, sv.to_device(p), out=yv)
    torch.cuda.synchronize()
    ref = oracle.forward(d, p, x)
    assert np.abs(yv.cpu().numpy() - ref).max() <= TOL


@pytest.mark.parametrize("HW", [(256, 256), (35, 129), (1, 5)])
def test_u8_within_one_lsb(sv, HW):
    import torch
    H, W = HW
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(9 + H, 1, H, W, d)
    x8 = si.to_u8(x)
    y8 = sv.apply(torch.from_numpy(x8).cuda(), sv.to_device(p))
    torch.cuda.synchronize()
    ref = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(x8)))
    diff = np.abs(y8.cpu().numpy().astype(int) - ref.astype(int))
    assert diff.max() <= 1
    assert (diff > 0).mean() < 1e-3


def test_deterministic(sv):
    d = si.spatial_dims(64, 256)
    x, p = si.make_batch(10, 2, 64, 256, d)
    a = run(sv, x, p)
    b = run(sv, x, p)
    assert np.array_equal(a, b)


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["mix"])
def test_4k_full_size(sv, mode):
    """The 3840x2160 bench workload, FP32, in the launch configuration the
    benchmark times, against the full oracle (OpenMP)."""
    H, W = 2160, 3840
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(1), 1, H, W, d, mode=mode)
    y = run(sv, x, p).astype(np.float64)
    ref = oracle.forward(d, p, x)
    assert np.abs(y - ref).max() <= TOL


def test_4k_u8_sampled_rows(sv):
    import torch
    H, W = 2160, 3840
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(1), 1, H, W, d)
    x8 = si.to_u8(x)
    y8 = sv.apply(torch.from_numpy(x8).cuda(), sv.to_device(p)).cpu().numpy()
    ref = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(x8)))
    diff = np.abs(y8.astype(int) - ref.astype(int))
    assert diff.max() <= 1


@pytest.mark.parametrize("ctas", [1, 7, 100, 152, 1000])
def test_cta_cap_gives_identical_output(sv, ctas):
    """svdlut_apply_cfg plans for a capped number of persistent CTAs; the
    per-pixel arithmetic, hence every output bit, is unchanged."""
    import torch
    H, W = 300, 517
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(9), 2, H, W, d)
    xt, pd = torch.from_numpy(x).cuda(), sv.to_device(p)
    ref = sv.apply(xt, pd)
    got = sv.apply(xt, pd, ctas=ctas)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_unaligned_factors_give_identical_output(sv):
    """Factors at 16-byte aligned addresses are copied to shared memory
    asynchronously; any other 4-byte aligned address takes the general
    loader.  Both compute (U S) w the same way: every output bit agrees."""
    import torch
    H, W = 120, 200
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(10), 2, H, W, d)
    xt, pd = torch.from_numpy(x).cuda(), sv.to_device(p)
    ref = sv.apply(xt, pd)
    shifted = dict(pd)
    for n in ("U", "V"):
        buf = torch.zeros(pd[n].numel() + 1, dtype=torch.float32, device="cuda")
        view = buf[1:].view(pd[n].shape)
        view.copy_(pd[n])
        shifted[n] = view
    got = sv.apply(xt, shifted)
    torch.cuda.synchronize()
    assert shifted["U"].data_ptr() % 16 != 0
    assert torch.equal(got, ref)
    assert np.abs(got.cpu().numpy().astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def _random_case(rng):
    """LUT dims over their whole range; grids at most one vertex per 4 pixels
    (the coarse spatial features of the method; denser slices of a 128-px
    tile need not fit in shared memory)."""
    D = int(rng.integers(2, 34))
    B, H, W = int(rng.integers(1, 4)), int(rng.integers(1, 300)), int(rng.integers(1, 300))
    d = si.Dims(D, int(rng.integers(1, D + 1)), int(rng.integers(0, 49)),
                int(rng.integers(2, max(3, min(64, W // 4) + 1))), int(rng.integers(2, max(3, min(64, H // 4) + 1))),
                int(rng.integers(2, 65)))
    return d, B, H, W


@pytest.mark.parametrize("seed", range(12))
def test_random_dims_and_sizes(sv, seed):
    """Seeded random transform dims and image sizes, F32 and u8, against the
    oracle."""
    import torch
    rng = np.random.default_rng(4000 + seed)
    d, B, H, W = _random_case(rng)
    x, p = si.make_batch(5000 + seed, B, H, W, d)
    pd = sv.to_device(p)
    y = sv.apply(torch.from_numpy(x).cuda(), pd).cpu().numpy().astype(np.float64)
    assert np.abs(y - oracle.forward(d, p, x)).max() <= TOL, (d, B, H, W)
    x8 = si.to_u8(x)
    y8 = sv.apply(torch.from_numpy(x8).cuda(), pd).cpu().numpy().astype(int)
    ref8 = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(x8))).astype(int)
    assert np.abs(y8 - ref8).max() <= 1, (d, B, H, W)


def test_8k_frame_u8_and_f32(sv):
    """A 7680x4320 frame (33 Mpx: beyond the 4K workload, for index widths)
    in FP32 and u8 against the oracle."""
    import torch
    H, W = 4320, 7680
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(11), 1, H, W, d)
    pd = sv.to_device(p)
    ref = oracle.forward(d, p, x)
    y = sv.apply(torch.from_numpy(x).cuda(), pd).cpu().numpy().astype(np.float64)
    assert np.abs(y - ref).max() <= TOL
    x8 = si.to_u8(x)
    y8 = sv.apply(torch.from_numpy(x8).cuda(), pd).cpu().numpy().astype(int)
    ref8 = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(x8))).astype(int)
    assert np.abs(y8 - ref8).max() <= 1


@pytest.mark.parametrize("dims", ["paper", "spatial"])
def test_on_vertex_and_upper_edge_inputs(sv, dims):
    """Inputs exactly on LUT and slicing vertices (p = i/32, which includes
    every i/16 of the 17-vertex intensity axis), at 0 and at the upper edge
    p = 1 (where the cell below is taken with frac = 1, reading R5), on an
    image whose pixel positions also fall on spatial vertices: 257 x 257, so
    (W-1) and (H-1) are multiples of (Ds-1) for Ds = 17 and for the
    1/8-resolution Ds = 33.  FP32 within 2e-5 of the oracle; the 8-bit codes
    0 and 255 (p = 0 and 1) within 1 LSB."""
    import torch
    H = W = 257
    d = si.paper_dims() if dims == "paper" else si.spatial_dims(H, W)
    assert (W - 1) % (d.Dsx - 1) == 0 and (H - 1) % (d.Dsy - 1) == 0
    rng = np.random.default_rng(31)
    _, p = si.make_batch(32, 2, H, W, d)
    x = (rng.integers(0, 33, size=(2, 3, H, W)) / 32.0).astype(np.float32)
    x[0, :, :64] = 1.0          # upper edge on every axis
    x[1, :, :64] = 0.0
    x[1, 0, 64:128] = 1.0       # mixed: one channel at the edge
    check_f32(sv, d, x, p)
    x8 = np.where(rng.uniform(size=x.shape) < 0.5, 0, 255).astype(np.uint8)
    y8 = sv.apply(torch.from_numpy(x8).cuda(), sv.to_device(p)).cpu().numpy().astype(int)
    ref = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(x8))).astype(int)
    assert np.abs(y8 - ref).max() <= 1


@pytest.mark.parametrize("d,B,H,W", [(si.spatial_dims(130, 515), 2, 130, 515), (si.paper_dims(), 3, 67, 257),
                                     (si.Dims(33, 33, 48, 9, 7, 64), 1, 70, 260), (si.Dims(2, 1, 0, 2, 2, 2), 2, 5, 9),
                                     (si.Dims(17, 8, 8, 9, 5, 33), 1, 300, 515)])
def test_workspace_path_equals_plain_path(sv, d, B, H, W):
    """svdlut_apply_ws (tables precomputed once per image into a workspace)
    against svdlut_apply (tables rebuilt in every CTA): identical bits, in
    FP32 and u8, and within 2e-5 of the oracle."""
    import torch
    x, p = si.make_batch(600 + H, B, H, W, d)
    xt, pd = torch.from_numpy(x).cuda(), sv.to_device(p)
    y_ws = sv.apply(xt, pd, workspace=True)
    y_plain = sv.apply(xt, pd, workspace=False)
    torch.cuda.synchronize()
    assert torch.equal(y_ws, y_plain)
    assert np.abs(y_ws.cpu().numpy().astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL
    x8 = torch.from_numpy(si.to_u8(x)).cuda()
    assert torch.equal(sv.apply(x8, pd, workspace=True), sv.apply(x8, pd, workspace=False))
    # an explicit workspace (stale contents do not matter) and the CTA cap
    from paper_2508_16121_gb300 import _lib
    need = _lib.load().svdlut_apply_workspace_size(ctypes_dims(sv, pd), B)
    ws = torch.full((need,), 0xAB, dtype=torch.uint8, device="cuda")
    assert torch.equal(sv.apply(xt, pd, workspace=ws, ctas=37), y_plain)


def ctypes_dims(sv, pd):
    import ctypes
    return ctypes.byref(sv.dims_of(pd))


def test_workspace_errors(sv):
    import ctypes
    import torch
    from paper_2508_16121_gb300 import _lib
    lib = _lib.load()
    d = si.spatial_dims(64, 128)
    x, p = si.make_batch(7, 1, 64, 128, d)
    xt, pd = torch.from_numpy(x).cuda(), sv.to_device(p)
    dims = sv.dims_of(pd)
    need = lib.svdlut_apply_workspace_size(ctypes.byref(dims), 1)
    assert need > 0 and lib.svdlut_apply_workspace_size(ctypes.byref(dims), 0) == 0
    with pytest.raises(ValueError):
        sv.apply(xt, pd, workspace=torch.empty(need - 1, dtype=torch.uint8, device="cuda"))
    ps = sv._param_struct(pd, 1, dims)
    y = torch.empty_like(xt)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    args = (ctypes.byref(dims), ctypes.byref(ps), 1, 64, 128, _lib.F32, ctypes.c_void_p(xt.data_ptr()),
            ctypes.c_void_p(y.data_ptr()), None)
    assert lib.svdlut_apply_ws(*args, None, need, None) == _lib.ERR_WORKSPACE
    assert lib.svdlut_apply_ws(*args, ctypes.c_void_p(buf.data_ptr()), need - 1, None) == _lib.ERR_WORKSPACE
    assert lib.svdlut_apply_ws(*args, ctypes.c_void_p(buf.data_ptr() + 4), need, None) == _lib.ERR_INVALID_ARG
    torch.cuda.synchronize()
