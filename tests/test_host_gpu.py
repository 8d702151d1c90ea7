"""svdlut_apply_host (host images, banded upload / transform / download on
overlapping streams) against svdlut_apply on the same data (bit-for-bit: the
same per-pixel arithmetic runs band by band) and against the FP64 oracle."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("B,H,W", [(1, 37, 130), (2, 300, 515), (1, 2160, 3840)])
def test_host_equals_device_apply(sv, B, H, W):
    import torch
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(5) + H, B, H, W, d)
    pd = sv.to_device(p)
    xh = torch.from_numpy(x).pin_memory()
    yh = sv.apply_host(xh, pd)
    ref = sv.apply(xh.cuda(), pd)
    torch.cuda.synchronize()
    assert torch.equal(yh, ref.cpu())


def test_host_u8_and_unpinned(sv):
    import torch
    H, W = 200, 333
    d = si.paper_dims()
    x, p = si.make_batch(si.config_seed(6), 1, H, W, d)
    pd = sv.to_device(p)
    xu = torch.from_numpy(si.to_u8(x))  # pageable: still correct, copies just do not overlap
    yu = sv.apply_host(xu, pd)
    torch.cuda.synchronize()
    assert torch.equal(yu, sv.apply(xu.cuda(), pd).cpu())


def test_host_matches_oracle(sv):
    import torch
    import oracle
    H, W = 130, 257
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(7), 1, H, W, d)
    yh = sv.apply_host(torch.from_numpy(x).pin_memory(), sv.to_device(p))
    torch.cuda.synchronize()
    ref = oracle.forward(d, p, x)
    assert np.abs(yh.numpy().astype(np.float64) - ref).max() <= 2e-5


def test_host_in_cuda_graph(sv):
    import torch
    H, W = 256, 384
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(8), 1, H, W, d)
    pd = sv.to_device(p)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    s = torch.cuda.Stream()
    sv.apply_host(xh, pd, out=yh, stream=s)  # first call outside capture (creates the copy streams)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sv.apply_host(xh, pd, out=yh, stream=s)
    yh.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(yh, sv.apply(xh.cuda(), pd).cpu())
