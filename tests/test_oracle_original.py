"""FP64 oracle of the paper's original (unfused) structure (Eqs. 7, 8, 5):
K spatial maps in full, the (K+3)->3 1x1 fusion conv, then the LUT transform
of the fused image.  Pinned against the fused-model oracle, which is pinned
on its own (test_oracle_forward.py):
- with the fusion conv the identity on X and zero on the maps, the result is
  the LUT transform of X alone (the fused model with K = 0);
- with identity LUT factors and the conv adding the maps of the grids that
  feed each channel, the result is the fused model's output (X plus the
  slices), as long as the fused image stays inside [0,1]."""
import numpy as np

import oracle
import svdlut_inputs as si


def fusion_matrix(K, maps=0.0, identity=1.0, bias=None):
    W = np.zeros((3, K + 3))
    for c in range(3):
        W[c, c] = identity
        for k in range(K):
            if k % 3 == c:
                W[c, 3 + k] = maps
    b = np.zeros(3) if bias is None else np.asarray(bias, dtype=np.float64)
    return np.concatenate([W.ravel(), b])


def test_identity_fusion_is_the_lut_transform_of_the_input():
    d = si.paper_dims()
    rng = np.random.default_rng(5)
    x = si.make_image(rng, 23, 41)
    p = si.make_params(rng, d)
    y = oracle.forward_original(d, p, fusion_matrix(d.K), x)
    d0 = si.Dims(d.D_t, d.rank, 0, 2, 2, 2)
    p0 = {k: v for k, v in p.items()}
    p0.update(g_xy=np.zeros((0, 2, 2)), g_xc=np.zeros((0, 2, 2)), g_yc=np.zeros((0, 2, 2)), grid_w=np.zeros((0, 4)))
    ref = oracle.forward(d0, p0, x)
    assert np.abs(y - ref).max() <= 1e-12


def test_identity_lut_and_summing_conv_is_the_fused_model():
    for d in (si.paper_dims(), si.spatial_dims(37, 29), si.Dims(9, 3, 5, 3, 4, 5)):
        rng = np.random.default_rng(7 + d.K)
        H, W = 37, 29
        x = 0.3 + 0.4 * si.make_image(rng, H, W)  # inside [0.3, 0.7]
        p = si.identity_params(d)
        p["g_xy"] = rng.uniform(-1, 1, p["g_xy"].shape)
        p["g_xc"] = rng.uniform(-1, 1, p["g_xc"].shape)
        p["g_yc"] = rng.uniform(-1, 1, p["g_yc"].shape)
        p["grid_w"] = rng.uniform(-0.02, 0.02, p["grid_w"].shape)
        fused = oracle.forward(d, p, x)
        assert fused.min() > 0.0 and fused.max() < 1.0  # no clamping of the fused image below
        y = oracle.forward_original(d, p, fusion_matrix(d.K, maps=1.0), x)
        assert np.abs(y - fused).max() <= 1e-12


def test_conv_bias_and_scale_reach_the_output_through_an_identity_lut():
    d = si.paper_dims()
    rng = np.random.default_rng(11)
    x = 0.25 + 0.5 * si.make_image(rng, 9, 13)
    p = si.identity_params(d)
    y = oracle.forward_original(d, p, fusion_matrix(d.K, identity=0.5, bias=[0.1, 0.2, 0.3]), x)
    assert np.abs(y - (0.5 * x + np.array([0.1, 0.2, 0.3])[:, None, None])).max() <= 1e-12


def test_planted_row_swap_of_the_conv_is_caught():
    d = si.paper_dims()
    rng = np.random.default_rng(13)
    x = si.make_image(rng, 11, 17)
    p = si.make_params(rng, d)
    f = rng.normal(0, 0.3, 3 * (d.K + 3) + 3)
    y = oracle.forward_original(d, p, f, x)
    g = f.copy()
    W = g[:3 * (d.K + 3)].reshape(3, d.K + 3)
    W[[0, 1]] = W[[1, 0]]
    assert np.abs(oracle.forward_original(d, p, g, x) - y).max() > 1e-3
