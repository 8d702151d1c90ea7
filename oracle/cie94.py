"""FP64 oracle of the colour-difference term of the training loss -- TEST
INFRASTRUCTURE (only tests/, __graft_entry__.smoke() and the benchmark's CPU
legs may use it).

The loss (Eq. 11) adds lambda_c = 0.005 times the distance between the
prediction and the ground truth in CIELAB under the CIE94 formula.  The paper
names the metric but not its conversion; the readings taken here are the
standard ones:
  - sRGB decoding (IEC 61966-2-1): lin = c / 12.92 for c <= 0.04045, else
    ((c + 0.055) / 1.055) ** 2.4, applied to the raw (unclamped) values;
  - linear sRGB -> XYZ by the matrix that maps the unit primaries to the sRGB
    primaries' chromaticities (0.64, 0.33), (0.30, 0.60), (0.15, 0.06) and the
    unit white to D65 (0.3127, 0.3290); derived here from those numbers;
  - CIELAB relative to that white, with the CIE constants eps = 216/24389 and
    kappa = 24389/27 for the linear part of f near zero;
  - CIE94 with the graphic-arts weights kL = kC = kH = 1, K1 = 0.045,
    K2 = 0.015, the ground truth as the reference (S_C = 1 + K1 C*_ref,
    S_H = 1 + K2 C*_ref), Delta H^2 = Delta a^2 + Delta b^2 - Delta C^2
    clamped at 0;
  - the loss is the mean of Delta E94 over pixels; its gradient is taken as 0
    where Delta E94 = 0.
Images are planar [..., 3, H, W] in [0,1] scale.
"""
from __future__ import annotations

import numpy as np

K1, K2 = 0.045, 0.015
EPS = 216.0 / 24389.0
KAPPA = 24389.0 / 27.0

# chromaticities of the sRGB primaries and of the D65 white
PRIMARIES = ((0.64, 0.33), (0.30, 0.60), (0.15, 0.06))
WHITE = (0.3127, 0.3290)


def _xyz_of(xy):
    x, y = xy
    return np.array([x / y, 1.0, (1.0 - x - y) / y])


def srgb_to_xyz_matrix():
    """Columns = XYZ of the primaries, scaled so that their sum is the white
    (the standard derivation from chromaticities)."""
    P = np.stack([_xyz_of(p) for p in PRIMARIES], axis=1)
    s = np.linalg.solve(P, _xyz_of(WHITE))
    return P * s[None, :]


def white_xyz():
    return _xyz_of(WHITE)


def srgb_decode(c):
    c = np.asarray(c, dtype=np.float64)
    return np.where(c <= 0.04045, c / 12.92, ((np.maximum(c, 0.04045) + 0.055) / 1.055) ** 2.4)


def _f(t):
    return np.where(t > EPS, np.cbrt(t), (KAPPA * t + 16.0) / 116.0)


def srgb_to_lab(x):
    """[..., 3, H, W] sRGB -> (L, a, b), each [..., H, W]."""
    x = np.asarray(x, dtype=np.float64)
    lin = srgb_decode(x)
    M = srgb_to_xyz_matrix()
    xyz = np.einsum("ij,...jhw->...ihw", M, lin)
    n = white_xyz()
    fx, fy, fz = (_f(xyz[..., i, :, :] / n[i]) for i in range(3))
    return 116.0 * fy - 16.0, 500.0 * (fx - fy), 200.0 * (fy - fz)


def delta_e94(lab_ref, lab):
    """CIE94 difference of lab from the reference lab_ref (tuples of arrays)."""
    L1, a1, b1 = lab_ref
    L2, a2, b2 = lab
    C1, C2 = np.hypot(a1, b1), np.hypot(a2, b2)
    dL, dC, da, db = L1 - L2, C1 - C2, a1 - a2, b1 - b2
    dH2 = np.maximum(da * da + db * db - dC * dC, 0.0)
    SC, SH = 1.0 + K1 * C1, 1.0 + K2 * C1
    return np.sqrt(dL * dL + (dC / SC) ** 2 + dH2 / SH ** 2)


def cie94_loss(y, target):
    """mean over pixels of Delta E94(Lab(target) -> Lab(y))."""
    return float(np.mean(delta_e94(srgb_to_lab(target), srgb_to_lab(y))))


def cie94_grad(y, target):
    """d cie94_loss / d y, by the chain rule through each step above."""
    y = np.asarray(y, dtype=np.float64)
    L1, a1, b1 = srgb_to_lab(target)
    # forward of the prediction, keeping the intermediates
    lin = srgb_decode(y)
    M = srgb_to_xyz_matrix()
    xyz = np.einsum("ij,...jhw->...ihw", M, lin)
    n = white_xyz()
    t = [xyz[..., i, :, :] / n[i] for i in range(3)]
    f = [_f(ti) for ti in t]
    L2, a2, b2 = 116.0 * f[1] - 16.0, 500.0 * (f[0] - f[1]), 200.0 * (f[1] - f[2])
    C1, C2 = np.hypot(a1, b1), np.hypot(a2, b2)
    dL, dC, da, db = L1 - L2, C1 - C2, a1 - a2, b1 - b2
    dH2raw = da * da + db * db - dC * dC
    SC, SH = 1.0 + K1 * C1, 1.0 + K2 * C1
    Q = dL * dL + (dC / SC) ** 2 + np.maximum(dH2raw, 0.0) / SH ** 2
    dE = np.sqrt(Q)
    # dQ / d(L2, a2, b2); C2 = |(a2, b2)|, dC2/da2 = a2 / C2 (0 at C2 = 0)
    safe = np.where(C2 > 0, C2, 1.0)
    ua, ub = np.where(C2 > 0, a2 / safe, 0.0), np.where(C2 > 0, b2 / safe, 0.0)
    hon = (dH2raw > 0).astype(np.float64)
    gL = -2.0 * dL
    ga = -2.0 * dC * ua / SC ** 2 + hon * (-2.0 * da + 2.0 * dC * ua) / SH ** 2
    gb = -2.0 * dC * ub / SC ** 2 + hon * (-2.0 * db + 2.0 * dC * ub) / SH ** 2
    scale = np.where(dE > 0, 0.5 / np.where(dE > 0, dE, 1.0), 0.0) / dE.size
    gL, ga, gb = gL * scale, ga * scale, gb * scale
    # through L = 116 fy - 16, a = 500 (fx - fy), b = 200 (fy - fz)
    gf = [500.0 * ga, 116.0 * gL - 500.0 * ga + 200.0 * gb, -200.0 * gb]
    dfdt = [np.where(ti > EPS, fi / (3.0 * np.where(ti > EPS, ti, 1.0)), KAPPA / 116.0) for ti, fi in zip(t, f)]
    gxyz = np.stack([gf[i] * dfdt[i] / n[i] for i in range(3)], axis=-3)
    glin = np.einsum("ij,...ihw->...jhw", M, gxyz)
    dlin = np.where(y <= 0.04045, 1.0 / 12.92,
                    2.4 / 1.055 * ((np.maximum(y, 0.04045) + 0.055) / 1.055) ** 1.4)
    return glin * dlin
