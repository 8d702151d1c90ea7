"""GPU parity of the CIE94 colour-difference loss term (Eq. 11) and of its
gradient (svdlut_cie94) against the FP64 oracle."""
import numpy as np
import pytest

import svdlut_inputs as si
from oracle import cie94 as ocie

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def _pair(seed, B, H, W, sigma=0.05):
    rng = np.random.default_rng(seed)
    t = np.stack([si.make_image(rng, H, W) for _ in range(B)]).astype(np.float32)
    y = (t + rng.normal(0, sigma, t.shape)).astype(np.float32)
    y[:, :, ::9, ::7] = rng.uniform(-0.2, 1.2, y[:, :, ::9, ::7].shape)  # outside [0,1]: raw values
    y[:, :, 1::11, 2::13] = t[:, :, 1::11, 2::13]  # identical pixels: zero difference, zero gradient
    return y, t


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("B,H,W", [(1, 1, 1), (2, 37, 53), (1, 64, 256)])
def test_loss_and_gradient_match_oracle(sv, B, H, W):
    import torch
    y, t = _pair(B * 100 + H, B, H, W)
    w = 0.005
    dy = torch.empty(y.shape, dtype=torch.float32, device="cuda")
    loss = float(sv.cie94(_cuda(y), _cuda(t), weight=w, dy=dy))
    ref = ocie.cie94_loss(y.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(ref, rel=1e-5, abs=1e-6)
    g = dy.cpu().numpy()
    gref = w * ocie.cie94_grad(y.astype(np.float64), t.astype(np.float64))
    assert np.abs(g - gref).max() <= 1e-3 * np.abs(gref).max() + 1e-12
    same = np.all(y == t, axis=1)
    assert np.all(g.transpose(0, 2, 3, 1)[same] == 0.0)


def test_accumulate_and_determinism(sv):
    import torch
    y, t = _pair(5, 2, 48, 80)
    yt, tt = _cuda(y), _cuda(t)
    d1 = torch.empty(y.shape, dtype=torch.float32, device="cuda")
    l1 = sv.cie94(yt, tt, weight=0.3, dy=d1)
    d2 = torch.full(y.shape, 1.5, dtype=torch.float32, device="cuda")
    l2 = sv.cie94(yt, tt, weight=0.3, dy=d2, accumulate=True)
    assert torch.equal(l1, l2)
    assert torch.equal(d2, d1 + 1.5)
    d3 = torch.empty_like(d1)
    sv.cie94(yt, tt, weight=0.3, dy=d3)
    assert torch.equal(d1, d3)
    assert float(sv.cie94(tt, tt)) == 0.0


def test_training_batch_size(sv):
    """The training batch (64 x 256 x 256): the loss against the oracle and
    the gradient on a sample of pixels."""
    import torch
    y, t = _pair(7, 64, 256, 256, sigma=0.03)
    dy = torch.empty(y.shape, dtype=torch.float32, device="cuda")
    loss = float(sv.cie94(_cuda(y), _cuda(t), weight=1.0, dy=dy))
    assert loss == pytest.approx(ocie.cie94_loss(y.astype(np.float64), t.astype(np.float64)), rel=1e-5)
    g = dy.cpu().numpy()
    rng = np.random.default_rng(8)
    for b in rng.integers(0, 64, 4):
        rows = slice(int(rng.integers(0, 240)), None)
        ys, ts = y[b:b + 1, :, rows, :16], t[b:b + 1, :, rows, :16]
        # the oracle gradient of a crop is the full-image gradient times crop / full pixel counts
        gref = ocie.cie94_grad(ys.astype(np.float64), ts.astype(np.float64)) * (ys[0, 0].size / (64 * 256 * 256))
        gs = g[b:b + 1, :, rows, :16]
        assert np.abs(gs - gref).max() <= 1e-3 * np.abs(gref).max()


def test_errors(sv):
    import torch
    from paper_2508_16121_gb300._lib import SvdlutError
    x = torch.zeros(1, 3, 4, 4, device="cuda")
    with pytest.raises(ValueError):
        sv.cie94(x, torch.zeros(1, 3, 4, 5, device="cuda"))
    with pytest.raises(SvdlutError):
        sv.cie94(x, x, ws=torch.empty(16, dtype=torch.uint8, device="cuda"))
