"""Pins of the FP64 oracle's forward map against what the paper and the
mathematics fix, independently of the oracle's own code.

- identity factors reproduce the input (bilinear interpolation is exact on
  affine functions, Supp. Eq. 15);
- a full-rank SVD of a dense table reproduces scipy's bilinear interpolation
  of that table (Eq. 9 + Supp. Eqs. 13-16);
- Eckart-Young fixes the rank-truncated reconstruction (Eq. 9, Sec. 3.2.2);
- the slicing term equals scipy's bilinear interpolation of each grid plane
  (Supp. Eqs. 17-21), with grid k feeding channel k mod 3 (Supp. Eq. 22);
- on-vertex queries return vertex values; continuity across cell edges;
  linearity in weights; clamping; degenerate W = 1 / H = 1.
Planted mistakes (operands swapped in the oracle's inputs) must fail the pins.
"""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
import svdlut_inputs as si

AX = ((0, 1), (0, 2), (1, 2))  # (alpha, beta) channels of rg, rb, gb


def rgi(table, pa, pb):
    """scipy bilinear interpolation of a [Da][Db] table on uniform [0,1] axes."""
    Da, Db = table.shape
    f = RegularGridInterpolator((np.linspace(0, 1, Da), np.linspace(0, 1, Db)), table,
                                method="linear")
    pts = np.stack([np.clip(pa, 0, 1).ravel(), np.clip(pb, 0, 1).ravel()], axis=-1)
    return f(pts).reshape(np.shape(pa))


def lut_only_params(rng, D, tables, K=0):
    """Full-rank factors of given dense tables [3][3][D][D] via numpy SVD."""
    U = np.zeros((3, 3, D, D))
    V = np.zeros((3, 3, D, D))
    S = np.zeros((3, 3, D))
    for c in range(3):
        for p in range(3):
            u, s, vt = np.linalg.svd(tables[c, p])
            U[c, p], S[c, p], V[c, p] = u, s, vt.T
    d = si.Dims(D, D, K, 5, 4, 6)
    return d, dict(U=U, S=S, V=V, lut_w=rng.uniform(-1, 1, (3, 4)),
                   g_xy=np.zeros((K, 4, 5)), g_xc=np.zeros((K, 5, 6)), g_yc=np.zeros((K, 4, 6)),
                   grid_w=np.zeros((K, 4)))


@pytest.mark.parametrize("dims", [si.paper_dims(), si.spatial_dims(37, 29), si.Dims(2, 1, 3, 2, 2, 2)])
@pytest.mark.parametrize("HW", [(1, 1), (1, 7), (5, 1), (23, 41)])
def test_identity_reproduces_input(dims, HW):
    rng = np.random.default_rng(1)
    x = si.make_image(rng, *HW)
    y = oracle.forward(dims, si.identity_params(dims), x)
    assert np.abs(y - x).max() <= 1e-15


@pytest.mark.parametrize("D", [2, 3, 17, 33])
def test_full_rank_svd_matches_scipy_bilinear(D):
    rng = np.random.default_rng(D)
    tables = rng.uniform(-1, 2, size=(3, 3, D, D))
    d, p = lut_only_params(rng, D, tables)
    x = rng.uniform(0, 1, size=(3, 9, 11))
    y = oracle.forward(d, p, x)
    for c in range(3):
        ref = p["lut_w"][c, 3] + sum(p["lut_w"][c, q] * rgi(tables[c, q], x[a], x[b])
                                     for q, (a, b) in enumerate(AX))
        assert np.abs(y[c] - ref).max() <= 1e-12


def test_planted_swap_of_u_and_v_is_caught():
    rng = np.random.default_rng(7)
    D = 9
    tables = rng.uniform(0, 1, size=(3, 3, D, D))
    d, p = lut_only_params(rng, D, tables)
    bad = dict(p, U=p["V"], V=p["U"])  # transposed operand
    x = rng.uniform(0, 1, size=(3, 6, 6))
    y = oracle.forward(d, bad, x)
    ref = p["lut_w"][0, 3] + sum(p["lut_w"][0, q] * rgi(tables[0, q], x[a], x[b])
                                 for q, (a, b) in enumerate(AX))
    assert np.abs(y[0] - ref).max() > 1e-3


@pytest.mark.parametrize("R", [1, 4, 8, 16])
def test_eckart_young_truncation(R):
    rng = np.random.default_rng(R)
    T = rng.uniform(0, 1, size=(33, 33))
    u, s, vt = np.linalg.svd(T)
    TR = oracle.lut_from_svd(u[:, :R], s[:R], vt[:R].T)
    assert abs(np.linalg.norm(T - TR) - np.sqrt((s[R:] ** 2).sum())) <= 1e-10
    full = oracle.lut_from_svd(u, s, vt.T)
    assert np.abs(full - T).max() <= 1e-12


def test_reconstruction_orientation():
    # rank 1: T[i][j] = u_i s v_j -- U indexes rows (first axis), V columns
    u = np.arange(1.0, 6.0)[:, None]
    v = np.array([1.0, 10.0, 100.0, 1000.0, 1e4])[:, None]
    T = oracle.lut_from_svd(u, [2.0], v)
    assert T[1, 0] == 4.0 and T[0, 1] == 20.0


@pytest.mark.parametrize("K", [1, 3, 6, 8])
def test_slicing_matches_scipy_per_plane(K):
    rng = np.random.default_rng(100 + K)
    d = si.Dims(5, 2, K, 7, 5, 9)
    p = si.make_params(rng, d)
    p = {k: v.astype(np.float64) for k, v in p.items()}
    p["lut_w"][:] = 0.0  # LUT term off
    H, W = 13, 17
    x = rng.uniform(0, 1, size=(3, H, W))
    y = oracle.forward(d, p, x)
    yy, xx = np.meshgrid(np.arange(H) / (H - 1), np.arange(W) / (W - 1), indexing="ij")
    ref = np.zeros((3, H, W))
    for k in range(K):
        c = k % 3
        w = p["grid_w"][k]
        ref[c] += (w[0] * rgi(p["g_xy"][k], yy, xx) + w[1] * rgi(p["g_xc"][k], xx, x[c])
                   + w[2] * rgi(p["g_yc"][k], yy, x[c]) + w[3])
    assert np.abs(y - ref).max() <= 1e-13


def test_planted_transposed_xy_plane_is_caught():
    rng = np.random.default_rng(5)
    d = si.Dims(3, 1, 1, 6, 6, 3)
    p = {k: v.astype(np.float64) for k, v in si.make_params(rng, d).items()}
    p["lut_w"][:] = 0.0
    p["grid_w"][0] = [1.0, 0.0, 0.0, 0.0]
    x = rng.uniform(0, 1, size=(3, 8, 10))
    good = oracle.forward(d, p, x)
    bad = oracle.forward(d, dict(p, g_xy=np.ascontiguousarray(p["g_xy"].transpose(0, 2, 1))), x)
    assert np.abs(good - bad).max() > 1e-3


def test_on_vertex_queries_return_vertex_values():
    rng = np.random.default_rng(3)
    d = si.paper_dims()
    p = {k: v.astype(np.float64) for k, v in si.make_params(rng, d).items()}
    H = W = 257  # x' = x/256 lands on grid vertices every 16 px
    idx = rng.integers(0, 33, size=(3, H, W))
    x = idx / 32.0
    y = oracle.forward(d, p, x)
    T = np.einsum("cpir,cpr,cpjr->cpij", p["U"], p["S"], p["V"])
    rows = np.arange(0, H, 16)
    cols = np.arange(0, W, 16)
    for c in range(3):
        for r in rows[:5]:
            for q in cols[:5]:
                v = p["lut_w"][c, 3] + sum(p["lut_w"][c, k] * T[c, k, idx[a, r, q], idx[b, r, q]]
                                           for k, (a, b) in enumerate(AX))
                for k in range(c, d.K, 3):
                    w = p["grid_w"][k]
                    jc = idx[c, r, q] // 2  # 33-vertex query on a 17-vertex axis
                    exact = idx[c, r, q] % 2 == 0
                    if not exact:
                        break
                    v += (w[0] * p["g_xy"][k, r // 16, q // 16] + w[1] * p["g_xc"][k, q // 16, jc]
                          + w[2] * p["g_yc"][k, r // 16, jc] + w[3])
                else:
                    assert abs(y[c, r, q] - v) <= 1e-12


def test_continuity_across_cell_edges():
    rng = np.random.default_rng(4)
    d = si.paper_dims()
    p = si.make_params(rng, d)
    i = rng.integers(1, 32, size=(3, 4, 4))
    xm = i / 32.0 - 1e-12
    xp = i / 32.0 + 1e-12
    ym, yp = oracle.forward(d, p, xm), oracle.forward(d, p, xp)
    assert np.abs(ym - yp).max() <= 1e-10


def test_linear_in_weights_and_grids():
    rng = np.random.default_rng(6)
    d = si.Dims(9, 3, 4, 5, 6, 7)
    p = {k: v.astype(np.float64) for k, v in si.make_params(rng, d).items()}
    x = rng.uniform(0, 1, size=(3, 7, 9))
    y0 = oracle.forward(d, p, x)
    for name in ("lut_w", "grid_w", "g_xy", "g_xc", "g_yc"):
        dp = rng.normal(size=p[name].shape)
        y1 = oracle.forward(d, dict(p, **{name: p[name] + dp}), x)
        y2 = oracle.forward(d, dict(p, **{name: p[name] + 2 * dp}), x)
        assert np.abs((y2 - y1) - (y1 - y0)).max() <= 1e-12


def test_clamping_and_degenerate_sizes():
    rng = np.random.default_rng(8)
    d = si.spatial_dims(1, 1)
    p = si.make_params(rng, d)
    x = rng.uniform(-0.5, 1.5, size=(3, 1, 6))
    y = oracle.forward(d, p, x)
    yc = oracle.forward(d, p, np.clip(x, 0, 1))
    assert np.array_equal(y, yc)
    # W = H = 1: x' = y' = 0 reads the first grid vertex row / column
    x1 = rng.uniform(0, 1, size=(3, 1, 1))
    y1 = oracle.forward(d, dict(p, grid_w=np.tile([1.0, 0, 0, 0], (d.K, 1)),
                                lut_w=np.zeros((3, 4))), x1)
    for c in range(3):
        assert abs(y1[c, 0, 0] - sum(p["g_xy"][k, 0, 0] for k in range(c, d.K, 3))) <= 1e-7


def test_separable_route_agrees():
    rng = np.random.default_rng(9)
    for d in (si.paper_dims(), si.spatial_dims(20, 30)):
        p = si.make_params(rng, d)
        x = si.make_image(rng, 20, 30)
        a = oracle.forward(d, p, x)
        b = oracle.forward(d, p, x, separable=True)
        assert np.abs(a - b).max() <= 1e-13


def test_batched_equals_per_image():
    x, p = si.make_batch(11, 3, 9, 14, si.spatial_dims(9, 14))
    yb = oracle.forward(si.spatial_dims(9, 14), p, x)
    for b in range(3):
        yi = oracle.forward(si.spatial_dims(9, 14), {k: v[b] for k, v in p.items()}, x[b])
        assert np.array_equal(yb[b], yi)


def test_u8_conversions():
    v = np.arange(256, dtype=np.uint8)
    assert np.array_equal(oracle.u8_to_unit(v), v / 255.0)
    # clamp, then round to nearest in FP64; 0.5 * 255 = 127.5 exactly (the
    # one exact half-integer code in [0, 1]) rounds to the even 128
    y = np.array([-0.1, 0.0, 0.3 / 255, 0.7 / 255, 0.2, 0.5, 254.4 / 255, 254.6 / 255, 1.0, 7.0])
    q = oracle.quantize_u8(y)
    assert list(q) == [0, 0, 0, 1, 51, 128, 254, 255, 255, 255]
