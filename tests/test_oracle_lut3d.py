"""FP64 oracle of the 3D LUT transform (Eq. 3) and of the best fit of a 3D
LUT by a sum of 2D LUTs (the hypothesis of Eq. 4), pinned by closed forms:
trilinear interpolation reproduces affine tables and vertex values; the fit
is the orthogonal projection onto sums of functions of two indices, so it is
exact on such sums, leaves a residual orthogonal to all of them, and is
idempotent."""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si


def test_identity_and_affine_tables_are_reproduced():
    rng = np.random.default_rng(1)
    x = si.make_image(rng, 19, 23)
    t = si.make_lut3d(rng, 17, "identity")
    assert np.abs(oracle.lut3d_apply(t, x) - x).max() <= 1e-14
    a = rng.normal(size=3)
    Bm = rng.normal(size=(3, 3))
    aff = a[:, None, None, None] + np.einsum("cd,dijk->cijk", Bm, t)
    ref = a[:, None, None] + np.einsum("cd,dhw->chw", Bm, x)
    assert np.abs(oracle.lut3d_apply(aff, x) - ref).max() <= 1e-12


def test_vertex_queries_return_vertex_values():
    D = 9
    rng = np.random.default_rng(2)
    t = rng.normal(size=(3, D, D, D))
    idx = rng.integers(0, D, (3, 5, 7))
    x = idx / (D - 1.0)
    y = oracle.lut3d_apply(t, x)
    for c in range(3):
        assert np.allclose(y[c], t[c][idx[0], idx[1], idx[2]], atol=1e-14)


def test_fit_is_exact_on_sums_of_pair_tables():
    D = 11
    rng = np.random.default_rng(3)
    f, g, h = rng.normal(size=(D, D)), rng.normal(size=(D, D)), rng.normal(size=(D, D))
    t = f[:, :, None] + g[:, None, :] + h[None, :, :]
    A, Bt, C, rms = oracle.lut3d_fit2d(t)
    assert rms <= 1e-12
    assert np.abs(A[:, :, None] + Bt[:, None, :] + C[None, :, :] - t).max() <= 1e-12


def test_residual_is_orthogonal_to_pair_tables_and_fit_is_idempotent():
    D = 13
    rng = np.random.default_rng(4)
    t = rng.normal(size=(D, D, D))
    A, Bt, C, rms = oracle.lut3d_fit2d(t)
    fit = A[:, :, None] + Bt[:, None, :] + C[None, :, :]
    res = t - fit
    assert rms == pytest.approx(np.sqrt(np.mean(res ** 2)), rel=1e-12)
    for _ in range(3):
        f, g, h = rng.normal(size=(D, D)), rng.normal(size=(D, D)), rng.normal(size=(D, D))
        q = f[:, :, None] + g[:, None, :] + h[None, :, :]
        assert abs(np.sum(res * q)) <= 1e-9 * np.sqrt(np.sum(res ** 2) * np.sum(q ** 2))
    A2, B2, C2, rms2 = oracle.lut3d_fit2d(fit)
    assert rms2 <= 1e-12


def test_photo_grade_has_a_three_way_part_and_the_fit_is_close():
    rng = np.random.default_rng(5)
    t = si.make_lut3d(rng, 33, "photo")
    rmss = [oracle.lut3d_fit2d(t[c])[3] for c in range(3)]
    assert all(1e-5 < r < 0.05 for r in rmss), rmss
