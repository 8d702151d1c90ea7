"""GPU parity of the paper's original, unfused structure
(svdlut_apply_original: spatial maps and the fused image through HBM, then
the LUT transform) against its FP64 oracle, and against the fused transform
where the two definitions coincide."""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def random_fusion(rng, K):
    W = rng.normal(0, 0.15, (3, K + 3))
    W[np.arange(3), np.arange(3)] += 1.0
    return np.concatenate([W.ravel(), rng.uniform(-0.05, 0.05, 3)])


@pytest.mark.parametrize("B,H,W,d", [(1, 1, 1, si.spatial_dims(1, 1)), (2, 37, 130, si.paper_dims()),
                                     (1, 67, 257, si.spatial_dims(67, 257)), (1, 45, 140, si.Dims(9, 3, 5, 3, 4, 5)),
                                     (1, 30, 40, si.Dims(33, 8, 0, 2, 2, 2))])
def test_original_matches_oracle(sv, B, H, W, d):
    import torch
    rng = np.random.default_rng(H * 7 + W)
    x, p = si.make_batch(17 + H, B, H, W, d)
    f = np.stack([random_fusion(rng, d.K) for _ in range(B)])
    y = sv.apply_original(torch.from_numpy(x).cuda(), sv.to_device(p), torch.from_numpy(f).float().cuda())
    torch.cuda.synchronize()
    ref = oracle.forward_original(d, p, f, x)
    assert np.abs(y.cpu().numpy().astype(np.float64) - ref).max() <= 2e-5


def test_original_4k_frame(sv):
    import torch
    H, W = 2160, 3840
    d = si.spatial_dims(H, W)
    rng = np.random.default_rng(3)
    x, p = si.make_batch(si.config_seed(1), 1, H, W, d)
    f = random_fusion(rng, d.K)
    y = sv.apply_original(torch.from_numpy(x).cuda(), sv.to_device(p), torch.from_numpy(f).float().cuda())
    torch.cuda.synchronize()
    ref = oracle.forward_original(d, p, f, x)
    assert np.abs(y.cpu().numpy().astype(np.float64) - ref).max() <= 2e-5


def test_identity_lut_and_summing_conv_equal_the_fused_transform(sv):
    import torch
    d = si.paper_dims()
    rng = np.random.default_rng(21)
    x = 0.3 + 0.4 * si.make_image(rng, 64, 96)
    p = si.identity_params(d)
    for k in ("g_xy", "g_xc", "g_yc"):
        p[k] = rng.uniform(-1, 1, p[k].shape)
    p["grid_w"] = rng.uniform(-0.02, 0.02, p["grid_w"].shape)
    W = np.zeros((3, d.K + 3))
    for c in range(3):
        W[c, c] = 1.0
        for k in range(d.K):
            if k % 3 == c:
                W[c, 3 + k] = 1.0
    f = np.concatenate([W.ravel(), np.zeros(3)])
    pd = sv.to_device(p)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    y_orig = sv.apply_original(xt, pd, torch.from_numpy(f).float().cuda())
    y_fused = sv.apply(xt, pd)
    torch.cuda.synchronize()
    assert torch.abs(y_orig - y_fused).max().item() <= 2e-5
