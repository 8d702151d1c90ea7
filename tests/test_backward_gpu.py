"""GPU parity of svdlut_backward (through the C ABI) against the FP64 oracle
adjoint and against central differences of the FP64 oracle forward.

Tolerances (the adjoint has no stated bar; these follow from FP32 sums of
O(1) terms over the image): parameter gradients ||d - ref|| <= 1e-4 ||ref||
and max-abs <= 1e-3 max|ref|; dx max-abs <= 1e-4 on pixels away from a
vertex (the slope is set-valued on a vertex).
"""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

pytestmark = pytest.mark.gpu

NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def gpu_backward(sv, x, p, dy):
    import torch
    g = sv.backward(torch.from_numpy(x).cuda(), sv.to_device(p), torch.from_numpy(dy).cuda())
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def off_vertex(x, d, eps=1e-4):
    """pixels whose three channels are away from every LUT and grid vertex"""
    ok = np.ones(x.shape[:-3] + x.shape[-2:], dtype=bool)
    for D in (d.D_t, d.Dsc):
        u = x * (D - 1)
        ok &= np.all((np.abs(u - np.rint(u)) > eps * (D - 1)) | (x <= 0) | (x >= 1), axis=-3)
    return ok


def compare(got, ref, d, x):
    for n in NAMES:
        a, r = got["d" + n], ref["d" + n]
        if r.size == 0:
            continue
        nr = np.linalg.norm(r)
        assert np.linalg.norm(a - r) <= 1e-4 * max(nr, 1e-30) + 1e-6, (n, np.linalg.norm(a - r), nr)
        assert np.abs(a - r).max() <= 1e-3 * np.abs(r).max() + 1e-6, n
    m = np.broadcast_to(off_vertex(x, d)[:, None], x.shape)
    diff = np.abs(got["dx"] - ref["dx"])
    assert diff[m].max() <= 1e-4, diff[m].max()


@pytest.mark.parametrize("HW", [(64, 64), (1, 1), (7, 1), (1, 9), (37, 130), (70, 260)])
def test_backward_matches_oracle_spatial_dims(sv, HW):
    H, W = HW
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(300 + H + W, 1, H, W, d)
    dy = si.make_upstream(301 + H, x.shape)
    got = gpu_backward(sv, x, p, dy)
    ref = oracle.backward(d, p, x, dy)
    compare(got, ref, d, x)


@pytest.mark.parametrize("d", [si.paper_dims(), si.Dims(2, 1, 3, 2, 2, 2), si.Dims(17, 8, 8, 9, 5, 33),
                               si.Dims(33, 33, 0, 2, 2, 2), si.Dims(9, 3, 7, 3, 4, 5),
                               si.Dims(33, 33, 48, 9, 7, 64)])  # largest sizes: yc through the warp scatter
def test_backward_dims_variants(sv, d):
    x, p = si.make_batch(310, 2, 45, 140, d)
    dy = si.make_upstream(311, x.shape)
    got = gpu_backward(sv, x, p, dy)
    ref = oracle.backward(d, p, x, dy)
    compare(got, ref, d, x)


def test_backward_clamped_inputs_and_misaligned_width(sv):
    d = si.spatial_dims(21, 51)
    rng = np.random.default_rng(312)
    x = rng.uniform(-0.3, 1.3, size=(1, 3, 21, 51)).astype(np.float32)
    p = si.stack_params([si.make_params(rng, d)])
    dy = si.make_upstream(313, x.shape)
    got = gpu_backward(sv, x, p, dy)
    ref = oracle.backward(d, p, x, dy)
    compare(got, ref, d, x)
    assert np.all(got["dx"][(x < 0) | (x > 1)] == 0.0)


def test_backward_is_bitwise_deterministic(sv):
    d = si.spatial_dims(96, 256)
    x, p = si.make_batch(314, 2, 96, 256, d, mode="smooth")
    dy = si.make_upstream(315, x.shape)
    a = gpu_backward(sv, x, p, dy)
    b = gpu_backward(sv, x, p, dy)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("want", [("dgrid_w",), ("dg_xy", "dg_yc"), ("dU", "dg_xc"), ("dx", "dlut_w", "dgrid_w")])
def test_backward_gradient_subsets_equal_the_full_call(sv, want):
    """Any subset of the gradients (the grid weights without the grid
    planes, planes without the weights, LUT and grid parts apart) gives the
    same bits as the call that asks for all of them."""
    import torch
    d = si.Dims(17, 8, 9, 12, 9, 17)
    x, p = si.make_batch(330, 2, 72, 100, d)
    dy = si.make_upstream(331, x.shape)
    xt, pt, gt = torch.from_numpy(x).cuda(), sv.to_device(p), torch.from_numpy(dy).cuda()
    full = sv.backward(xt, pt, gt)
    part = sv.backward(xt, pt, gt, want=want)
    torch.cuda.synchronize()
    assert set(part) == set(want)
    for k in want:
        assert torch.equal(part[k], full[k]), k


def test_backward_matches_fp64_central_differences(sv):
    """directional derivatives of the FP64 oracle forward on a 64x64 crop"""
    d = si.spatial_dims(64, 64)
    x, p = si.make_batch(316, 1, 64, 64, d)
    x = np.clip(x, 0.01, 0.99).astype(np.float32)
    dy = si.make_upstream(317, x.shape)
    got = gpu_backward(sv, x, p, dy)
    pd = {k: v[0].astype(np.float64) for k, v in p.items()}
    rng = np.random.default_rng(318)
    h = 1e-6
    for n in NAMES:
        dirn = rng.standard_normal(pd[n].shape)
        fp = oracle.forward(d, dict(pd, **{n: pd[n] + h * dirn}), x[0])
        fm = oracle.forward(d, dict(pd, **{n: pd[n] - h * dirn}), x[0])
        fd = ((fp - fm) * dy[0]).sum() / (2 * h)
        an = (got["d" + n][0] * dirn).sum()
        assert abs(fd - an) <= 2e-4 * max(1.0, abs(fd)), (n, fd, an)


def test_autograd_function(sv):
    import torch
    d = si.spatial_dims(32, 48)
    x, p = si.make_batch(319, 1, 32, 48, d)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    pt = {k: v.requires_grad_(True) for k, v in sv.to_device(p).items()}
    y = sv.apply_autograd(xt, pt)
    dy = torch.from_numpy(si.make_upstream(320, x.shape)).cuda()
    (y * dy).sum().backward()
    ref = oracle.backward(d, p, x, dy.cpu().numpy())
    assert np.abs(pt["U"].grad.cpu().numpy() - ref["dU"]).max() <= 1e-3 * np.abs(ref["dU"]).max()
    m = np.broadcast_to(off_vertex(x, d)[:, None], x.shape)
    assert np.abs(xt.grad.cpu().numpy() - ref["dx"])[m].max() <= 1e-4


def test_workspace_errors(sv):
    import ctypes
    import torch
    from paper_2508_16121_gb300 import _lib
    d = si.spatial_dims(16, 16)
    x, p = si.make_batch(321, 1, 16, 16, d)
    xt = torch.from_numpy(x).cuda()
    pt = sv.to_device(p)
    dims = sv.dims_of(pt)
    ps = sv._param_struct(pt, 1, dims)
    dU = torch.empty_like(pt["U"])
    g = _lib.Grads(dU=dU.data_ptr())
    lib = _lib.load()
    need = lib.svdlut_backward_workspace_size(ctypes.byref(dims), 1, 16, 16)
    assert need > 0
    st = lib.svdlut_backward(ctypes.byref(dims), ctypes.byref(ps), 1, 16, 16, ctypes.c_void_p(xt.data_ptr()),
                             ctypes.c_void_p(xt.data_ptr()), None, ctypes.byref(g), None, 0, None)
    assert st == _lib.ERR_WORKSPACE


@pytest.mark.slow
def test_backward_1080p_batch_of_8(sv):
    """the benchmarked adjoint workload (8 x 1920x1080): image 0 against the
    full oracle, and linearity in dy over the whole batch"""
    import torch
    H, W, B = 1080, 1920, 8
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(3), B, H, W, d)
    dy1 = si.make_upstream(322, x.shape)
    dy2 = si.make_upstream(323, x.shape)
    g1 = gpu_backward(sv, x, p, dy1)
    ref = oracle.backward(d, {k: v[:1] for k, v in p.items()}, x[:1], dy1[:1])
    compare({k: v[:1] for k, v in g1.items()}, ref, d, x[:1])
    g2 = gpu_backward(sv, x, p, dy2)
    g12 = gpu_backward(sv, x, p, (dy1 + dy2).astype(np.float32))
    for k in g1:
        s = g1[k] + g2[k]
        assert np.abs(g12[k] - s).max() <= 1e-4 * max(np.abs(s).max(), 1.0), k


@pytest.mark.parametrize("seed", range(6))
def test_backward_random_dims_and_sizes(sv, seed):
    """Seeded random transform dims (grids at most one vertex per 8 pixels,
    as the method's low-resolution features, and at most 33 intensity
    vertices) and image sizes against the oracle adjoint."""
    rng = np.random.default_rng(6000 + seed)
    D = int(rng.integers(2, 34))
    B, H, W = int(rng.integers(1, 3)), int(rng.integers(1, 160)), int(rng.integers(1, 200))
    d = si.Dims(D, int(rng.integers(1, D + 1)), int(rng.integers(0, 49)),
                int(rng.integers(2, max(3, min(64, W // 8) + 1))), int(rng.integers(2, max(3, min(64, H // 8) + 1))),
                int(rng.integers(2, 34)))
    x, p = si.make_batch(7000 + seed, B, H, W, d)
    dy = si.make_upstream(7100 + seed, x.shape)
    compare(gpu_backward(sv, x, p, dy), oracle.backward(d, p, x, dy), d, x)
