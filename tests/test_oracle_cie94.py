"""Pins of the FP64 oracle of the CIE94 colour-difference loss term (Eq. 11,
lambda_c = 0.005): the sRGB -> XYZ matrix against the 4-digit matrix of
IEC 61966-2-1, the CIELAB coordinates of white, black, greys and of the
sRGB primaries against their tabulated values, the CIE94 formula against its
closed forms for pure lightness, chroma and hue differences, and the
gradient against central differences."""
import math

import numpy as np
import pytest

from oracle import cie94


def _px(*rgb):
    return np.array(rgb, dtype=np.float64).reshape(3, 1, 1)


def _lab(*rgb):
    return tuple(float(v[0, 0]) for v in cie94.srgb_to_lab(_px(*rgb)))


def test_matrix_matches_the_standard():
    iec = np.array([[0.4124, 0.3576, 0.1805], [0.2126, 0.7152, 0.0722], [0.0193, 0.1192, 0.9505]])
    M = cie94.srgb_to_xyz_matrix()
    assert np.abs(M - iec).max() <= 6e-5
    assert np.allclose(M.sum(axis=1), cie94.white_xyz(), atol=1e-14)
    assert M[1].sum() == pytest.approx(1.0, abs=1e-14)


def test_decoding_endpoints_and_branch_point():
    d = cie94.srgb_decode(np.array([0.0, 1.0, 0.04045, 0.04045 + 1e-12]))
    assert d[0] == 0.0 and d[1] == pytest.approx(1.0, abs=1e-15)
    assert abs(d[2] - d[3]) <= 1e-8  # the two branches meet at 0.04045


def test_white_black_and_greys():
    assert _lab(1, 1, 1) == pytest.approx((100.0, 0.0, 0.0), abs=1e-12)
    assert _lab(0, 0, 0) == pytest.approx((0.0, 0.0, 0.0), abs=1e-12)
    Ls = []
    for g in np.linspace(0.0, 1.0, 11):
        L, a, b = _lab(g, g, g)
        assert abs(a) <= 1e-10 and abs(b) <= 1e-10
        Ls.append(L)
    assert np.all(np.diff(Ls) > 0)
    assert _lab(0.5, 0.5, 0.5)[0] == pytest.approx(53.389, abs=1e-3)


def test_primaries_match_their_tabulated_lab():
    # CIELAB (D65) of the sRGB primaries as tabulated in colour references
    # (computed there with the 4-digit matrix, hence the 0.01 tolerance)
    table = {(1, 0, 0): (53.2408, 80.0925, 67.2032), (0, 1, 0): (87.7347, -86.1827, 83.1793),
             (0, 0, 1): (32.2970, 79.1875, -107.8602)}
    for rgb, lab in table.items():
        assert _lab(*rgb) == pytest.approx(lab, abs=0.01)


def _lab_point(L, C, h):
    return (np.array([L]), np.array([C * math.cos(h)]), np.array([C * math.sin(h)]))


def test_cie94_closed_forms():
    # pure lightness difference: Delta E = |Delta L|
    assert cie94.delta_e94(_lab_point(60, 30, 1.0), _lab_point(52.5, 30, 1.0))[0] == pytest.approx(7.5, abs=1e-12)
    # pure chroma difference along one hue: Delta C / (1 + K1 C_ref); asymmetric in the reference
    assert cie94.delta_e94(_lab_point(50, 50, 0.3), _lab_point(50, 40, 0.3))[0] == pytest.approx(10 / 3.25, abs=1e-12)
    assert cie94.delta_e94(_lab_point(50, 40, 0.3), _lab_point(50, 50, 0.3))[0] == pytest.approx(10 / 2.8, abs=1e-12)
    # pure hue rotation by theta at chroma C: 2 C sin(theta / 2) / (1 + K2 C)
    th = 0.2
    want = 2 * 50 * math.sin(th / 2) / (1 + 0.015 * 50)
    assert cie94.delta_e94(_lab_point(50, 50, 0.7), _lab_point(50, 50, 0.7 + th))[0] == pytest.approx(want, abs=1e-12)
    # identical colours
    assert cie94.delta_e94(_lab_point(40, 20, 2.0), _lab_point(40, 20, 2.0))[0] == 0.0


def test_identical_images_have_zero_loss_and_gradient():
    rng = np.random.default_rng(1)
    t = rng.uniform(0, 1, (2, 3, 4, 5))
    assert cie94.cie94_loss(t, t) == 0.0
    assert np.all(cie94.cie94_grad(t, t) == 0.0)


@pytest.mark.parametrize("seed", [2, 3])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 1, (1, 3, 3, 4))
    y = t + rng.normal(0, 0.1, t.shape)
    y[0, :, 0, 0] = [-0.05, 0.02, 1.1]  # both decoding branches and values outside [0,1]
    g = cie94.cie94_grad(y, t)
    h = 1e-6
    num = np.zeros_like(y)
    for idx in np.ndindex(y.shape):
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        num[idx] = (cie94.cie94_loss(yp, t) - cie94.cie94_loss(ym, t)) / (2 * h)
    assert np.abs(g - num).max() <= 1e-6 * max(1.0, np.abs(num).max())
