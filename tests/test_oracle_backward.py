"""Pins of the FP64 oracle's adjoint: central finite differences of the
oracle's forward map (a different code path) in FP64.

The transform is linear in the LUT weights and in every grid plane and grid
weight, and linear in each of U, S and V separately (Eq. 9), so central
differences along those directions are exact up to rounding.  In the pixel
values it is piecewise bilinear (Supp. Eq. 15): differences are exact away
from cell edges, so pixels within 1e-4 of a vertex are kept out of the
pixel-gradient check.
"""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")


def setup(seed, d, H, W):
    rng = np.random.default_rng(seed)
    p = {k: v.astype(np.float64) for k, v in si.make_params(rng, d).items()}
    x = rng.uniform(0.02, 0.98, size=(3, H, W))
    dy = rng.standard_normal(size=(3, H, W))
    return rng, p, x, dy


@pytest.mark.parametrize("d", [si.Dims(9, 3, 4, 5, 6, 7), si.paper_dims(), si.Dims(2, 2, 8, 2, 3, 2)])
def test_parameter_gradients_match_central_differences(d):
    rng, p, x, dy = setup(21, d, 11, 13)
    g = oracle.backward(d, p, x, dy)
    h = 1e-6
    for name in NAMES:
        for _ in range(3):
            dirn = rng.standard_normal(size=p[name].shape)
            fp = oracle.forward(d, dict(p, **{name: p[name] + h * dirn}), x)
            fm = oracle.forward(d, dict(p, **{name: p[name] - h * dirn}), x)
            fd = ((fp - fm) * dy).sum() / (2 * h)
            an = (g["d" + name] * dirn).sum()
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (name, fd, an)


def test_pixel_gradient_matches_central_differences_off_vertex():
    d = si.spatial_dims(12, 10)
    rng, p, x, dy = setup(22, d, 12, 10)
    g = oracle.backward(d, p, x, dy)
    h = 1e-7
    checked = 0
    for c in range(3):
        for r in range(12):
            for q in range(10):
                v = x[c, r, q]
                near = min(abs(v * 32 - round(v * 32)), abs(v * 16 - round(v * 16)))
                if near < 1e-4 * 32:
                    continue
                xp, xm = x.copy(), x.copy()
                xp[c, r, q] += h
                xm[c, r, q] -= h
                fd = ((oracle.forward(d, p, xp) - oracle.forward(d, p, xm)) * dy).sum() / (2 * h)
                assert abs(fd - g["dx"][c, r, q]) <= 1e-6 * max(1.0, abs(fd))
                checked += 1
    assert checked > 300


def test_pixel_gradient_zero_outside_unit_range():
    d = si.Dims(5, 2, 3, 3, 3, 3)
    rng, p, x, dy = setup(23, d, 3, 4)
    x[0, 0, 0], x[1, 1, 1], x[2, 2, 2] = -0.3, 1.2, 0.5
    g = oracle.backward(d, p, x, dy)
    assert g["dx"][0, 0, 0] == 0.0 and g["dx"][1, 1, 1] == 0.0


def test_bias_gradients_are_sums_of_upstream():
    d = si.Dims(5, 2, 7, 3, 4, 5)
    rng, p, x, dy = setup(24, d, 6, 5)
    g = oracle.backward(d, p, x, dy)
    for c in range(3):
        assert abs(g["dlut_w"][c, 3] - dy[c].sum()) <= 1e-12
    for k in range(d.K):
        assert abs(g["dgrid_w"][k, 3] - dy[k % 3].sum()) <= 1e-12


def test_batched_gradients_are_per_image():
    d = si.Dims(5, 2, 3, 3, 3, 3)
    x, p = si.make_batch(25, 2, 4, 5, d)
    dy = si.make_upstream(26, x.shape)
    gb = oracle.backward(d, p, x, dy)
    for b in range(2):
        gi = oracle.backward(d, {k: v[b] for k, v in p.items()}, x[b], dy[b])
        for k in gi:
            assert np.array_equal(gb[k][b], gi[k])
