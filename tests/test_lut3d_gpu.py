"""GPU parity of the 3D LUT transform (Eq. 3, svdlut_lut3d_apply) and of the
best fit of a 3D LUT by a sum of 2D LUTs (the hypothesis of Eq. 4,
svdlut_lut3d_fit2d) against their FP64 oracles, and of the fitted tables run
through the 2D transform."""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _images(seed, B, H, W, spill=False):
    rng = np.random.default_rng(seed)
    x = np.stack([si.make_image(rng, H, W) for _ in range(B)])
    if spill:  # values outside [0,1] are clamped before the lookup
        x[:, :, ::7, ::5] = rng.uniform(-0.5, 1.5, x[:, :, ::7, ::5].shape)
    return x


@pytest.mark.parametrize("B,H,W,D,kinds", [(1, 1, 1, 33, ["photo"]), (2, 37, 131, 33, ["photo", "smooth"]),
                                           (3, 64, 96, 9, ["smooth", "photo", "identity"]),
                                           (1, 5, 7, 2, ["photo"])])
def test_lut3d_apply_matches_oracle(sv, B, H, W, D, kinds):
    rng = np.random.default_rng(1000 + H + D)
    lut = np.stack([si.make_lut3d(rng, D, k) for k in kinds])
    x = _images(H * 3 + W, B, H, W, spill=True)
    y = sv.lut3d_apply(_cuda(x), _cuda(lut)).cpu().numpy()
    ref = oracle.lut3d_apply(lut, x)
    assert np.abs(y - ref).max() <= TOL


def test_lut3d_apply_shared_table_and_identity(sv):
    rng = np.random.default_rng(5)
    x = _images(6, 2, 40, 44, spill=True)
    y = sv.lut3d_apply(_cuda(x), _cuda(si.make_lut3d(rng, 33, "identity"))).cpu().numpy()
    assert np.abs(y - np.clip(x, 0.0, 1.0)).max() <= 1e-6


def test_lut3d_apply_4k_frame(sv):
    rng = np.random.default_rng(7)
    lut = si.make_lut3d(rng, 33, "photo")
    x = _images(si.config_seed(1), 1, 2160, 3840)
    y = sv.lut3d_apply(_cuda(x), _cuda(lut)).cpu().numpy()
    assert np.abs(y - oracle.lut3d_apply(lut, x)).max() <= TOL


@pytest.mark.parametrize("D,kind", [(33, "photo"), (33, "smooth"), (17, "photo"), (2, "smooth")])
def test_fit2d_matches_oracle(sv, D, kind):
    rng = np.random.default_rng(D * 13 + len(kind))
    lut = np.stack([si.make_lut3d(rng, D, kind), si.make_lut3d(rng, D, "photo")])
    tables, rms = sv.lut3d_fit2d(_cuda(lut))
    tables, rms = tables.cpu().numpy(), rms.cpu().numpy()
    for b in range(2):
        for c in range(3):
            A, Bt, C, r = oracle.lut3d_fit2d(lut[b, c])
            assert np.abs(tables[b, c, 0] - A).max() <= TOL
            assert np.abs(tables[b, c, 1] - Bt).max() <= TOL
            assert np.abs(tables[b, c, 2] - C).max() <= TOL
            assert abs(rms[b, c] - r) <= 1e-5 + 1e-4 * r


def test_fit_of_a_2d_sum_is_exact(sv):
    rng = np.random.default_rng(8)
    D = 33
    A, Bt, C = (rng.uniform(-0.3, 0.3, (3, D, D)) for _ in range(3))
    t = A[:, :, :, None] + Bt[:, :, None, :] + C[:, None, :, :]
    _, rms = sv.lut3d_fit2d(_cuda(t))
    assert rms.abs().max().item() <= 1e-6


def test_fitted_tables_through_the_2d_transform(sv):
    """Trilinear interpolation of A[r][g] + Bt[r][b] + C[g][b] is the sum of
    the bilinear interpolations of A, Bt and C, so the 2D transform of the
    fitted tables equals the 3D transform of the fitted 3D table."""
    import torch
    rng = np.random.default_rng(9)
    D, B, H, W = 33, 2, 45, 70
    lut = np.stack([si.make_lut3d(rng, D, "photo"), si.make_lut3d(rng, D, "smooth")])
    tables, _ = sv.lut3d_fit2d(_cuda(lut))
    x = _images(10, B, H, W, spill=True)
    y2d = sv.apply(_cuda(x), sv.fit_params(tables))
    torch.cuda.synchronize()
    tb = tables.cpu().numpy().astype(np.float64)
    fit3d = (tb[:, :, 0, :, :, None] + tb[:, :, 1, :, None, :] + tb[:, :, 2, None, :, :])
    ref = oracle.lut3d_apply(fit3d, x)
    assert np.abs(y2d.cpu().numpy() - ref).max() <= 2e-5


def test_lut3d_errors(sv):
    import torch
    from paper_2508_16121_gb300._lib import SvdlutError
    x = torch.zeros(1, 3, 4, 4, device="cuda")
    with pytest.raises(SvdlutError):
        sv.lut3d_apply(x, torch.zeros(1, 3, 34, 34, 34, device="cuda"))
    with pytest.raises(SvdlutError):
        sv.lut3d_fit2d(torch.zeros(1, 3, 1, 1, 1, device="cuda"))
    import ctypes
    from paper_2508_16121_gb300 import _lib
    t = torch.zeros(1, 3, 5, 5, 5, device="cuda")
    y = torch.empty_like(x)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    lib = _lib.load()
    st = lib.svdlut_lut3d_apply(5, ctypes.c_void_p(t.data_ptr()), 1, 4, 4, ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(ws.data_ptr()), 16, None)
    assert st == 4  # SVDLUT_ERR_WORKSPACE
