"""Seeded synthetic inputs for SVDLUT apply, adjoint and generator workloads.

This module only draws numbers; it holds none of the method's arithmetic
(no interpolation, no factor product, no slicing).  Both the CPU oracle
tests and the CUDA path tests/bench take their inputs from here.

Stand-ins: the paper evaluates on FiveK / PPR10K photographs (Sec. 4.1,
480p to full resolution).  Those are not available, so images are
synthetic: 64x64 tiles alternate checkerboard-wise between i.i.d.
U(0,1) noise (incoherent lookups) and smooth seeded gradients (coherent
lookups, photo-like).

Layouts (all C-contiguous, float32 unless stated):
  image   [3][H][W]                       planar RGB in [0,1]
  U, V    [3 c][3 pair][D_t][rank]        pair order (rg, rb, gb)
  S       [3 c][3 pair][rank]
  lut_w   [3 c][4]                        (w_rg, w_rb, w_gb, b)
  g_xy    [K][Dsy][Dsx]
  g_xc    [K][Dsx][Dsc]
  g_yc    [K][Dsy][Dsc]
  grid_w  [K][4]                          (w_xy, w_xc, w_yc, b)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 16121
PARAM_NAMES = ("U", "S", "V", "lut_w", "g_xy", "g_xc", "g_yc", "grid_w")
BATCH_SIZES = ((640, 480), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


@dataclass(frozen=True)
class Dims:
    """Grid sizes of one image's transform: LUT vertices per axis, SVD rank,
    number of 2D bilateral grids and grid vertices along x, y and intensity."""
    D_t: int = 33
    rank: int = 8
    K: int = 8
    Dsx: int = 17
    Dsy: int = 17
    Dsc: int = 17

    def as_tuple(self):
        return (self.D_t, self.rank, self.K, self.Dsx, self.Dsy, self.Dsc)


def paper_dims() -> Dims:
    """The paper's setting: D_t=33, N_s=8, K=6 grids of 17 vertices per axis."""
    return Dims(33, 8, 6, 17, 17, 17)


def spatial_dims(H: int, W: int, D_t: int = 33, rank: int = 8, K: int = 8, Dsc: int = 17) -> Dims:
    """Spatial features at 1/8 resolution: K=8 grids with ceil(W/8) x ceil(H/8)
    spatial vertices (at least 2 per axis) and 17 intensity vertices."""
    return Dims(D_t, rank, K, max(2, math.ceil(W / 8)), max(2, math.ceil(H / 8)), Dsc)


def image_seed(j: int) -> int:
    return SEED_BASE * 100 + j


def config_seed(i: int) -> int:
    return SEED_BASE + i


def make_image(rng: np.random.Generator, H: int, W: int, tile: int = 64,
               mode: str = "mix") -> np.ndarray:
    """Planar float32 [3][H][W] in [0,1].  mode: 'mix' (checkerboard of noise
    and smooth tiles), 'noise' or 'smooth'."""
    yy = (np.arange(H, dtype=np.float64)[:, None] / max(H, 1))
    xx = (np.arange(W, dtype=np.float64)[None, :] / max(W, 1))
    smooth = np.empty((3, H, W), dtype=np.float64)
    for c in range(3):
        a, bx, by = rng.uniform(0.1, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4)
        s = a + bx * xx + by * yy
        for _ in range(2):
            amp = rng.uniform(0.05, 0.25)
            fx, fy = rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0)
            ph = rng.uniform(0, 2 * math.pi)
            s = s + amp * np.sin(2 * math.pi * (fx * xx + fy * yy) + ph)
        smooth[c] = s
    smooth = np.clip(smooth, 0.0, 1.0)
    noise = rng.uniform(0.0, 1.0, size=(3, H, W))
    if mode == "smooth":
        out = smooth
    elif mode == "noise":
        out = noise
    else:
        ty = (np.arange(H)[:, None] // tile)
        tx = (np.arange(W)[None, :] // tile)
        is_noise = ((tx + ty) % 2 == 0)
        out = np.where(is_noise[None], noise, smooth)
    return np.ascontiguousarray(out.astype(np.float32))


def to_u8(img: np.ndarray) -> np.ndarray:
    """8-bit version of a [0,1] image: round(x*255)."""
    return np.ascontiguousarray(np.rint(np.clip(img, 0, 1) * 255.0).astype(np.uint8))


def to_u16(img: np.ndarray) -> np.ndarray:
    """16-bit version of a [0,1] image: round(x*65535)."""
    return np.round(np.clip(img, 0.0, 1.0) * 65535.0).astype(np.uint16)


def make_image_u16(rng: np.random.Generator, H: int, W: int, mode: str = "mix") -> np.ndarray:
    """Planar 16-bit codes [3][H][W] standing in for the 16-bit photo inputs
    (linear light, so most codes are dark): make_image raised to 2.2."""
    return to_u16(make_image(rng, H, W, mode=mode).astype(np.float64) ** 2.2)


def to_hwc(img: np.ndarray) -> np.ndarray:
    """Interleaved copy [..][H][W][3] of a planar image [..][3][H][W]."""
    return np.ascontiguousarray(np.moveaxis(img, -3, -1))


def identity_params(d: Dims, dtype=np.float64) -> dict:
    """Factors whose transform is the identity, with all grid terms off.

    Channel r is axis alpha of pairs rg and rb, g is axis beta of rg and
    alpha of gb, b is axis beta of rb and gb.  A table that equals its
    alpha coordinate is u0 = vertex coordinates, v0 = 1; one equal to its
    beta coordinate is u0 = 1, v0 = vertex coordinates.  Each channel is
    split evenly over the two pairs that contain it (weights 1/2)."""
    D, R = d.D_t, d.rank
    ramp = np.linspace(0.0, 1.0, D)
    ones = np.ones(D)
    U = np.zeros((3, 3, D, R))
    V = np.zeros((3, 3, D, R))
    S = np.zeros((3, 3, R))
    lut_w = np.zeros((3, 4))
    # (channel, pair, table follows alpha?)
    uses = {0: ((0, True), (1, True)), 1: ((0, False), (2, True)), 2: ((1, False), (2, False))}
    for c, lst in uses.items():
        for p, follows_alpha in lst:
            U[c, p, :, 0] = ramp if follows_alpha else ones
            V[c, p, :, 0] = ones if follows_alpha else ramp
            S[c, p, 0] = 1.0
            lut_w[c, p] = 0.5
    K = d.K
    return dict(U=U.astype(dtype), S=S.astype(dtype), V=V.astype(dtype), lut_w=lut_w.astype(dtype),
                g_xy=np.zeros((K, d.Dsy, d.Dsx), dtype), g_xc=np.zeros((K, d.Dsx, d.Dsc), dtype),
                g_yc=np.zeros((K, d.Dsy, d.Dsc), dtype), grid_w=np.zeros((K, 4), dtype))


def make_params(rng: np.random.Generator, d: Dims, sigma: float = 0.1) -> dict:
    """Per-image factors around the identity: U, V = identity + N(0, sigma);
    s = (1, U(0,1) x (rank-1)); LUT weights = identity + U(-0.05, 0.05),
    biases U(-0.02, 0.02); grid planes U(0,1), grid weights and biases
    U(-0.05, 0.05).  float32."""
    p = identity_params(d)
    D, R, K = d.D_t, d.rank, d.K
    U = p["U"] + rng.normal(0.0, sigma, size=(3, 3, D, R))
    V = p["V"] + rng.normal(0.0, sigma, size=(3, 3, D, R))
    S = np.empty((3, 3, R))
    S[..., 0] = 1.0
    if R > 1:
        S[..., 1:] = rng.uniform(0.0, 1.0, size=(3, 3, R - 1))
    lut_w = p["lut_w"].copy()
    lut_w[:, :3] += rng.uniform(-0.05, 0.05, size=(3, 3))
    lut_w[:, 3] = rng.uniform(-0.02, 0.02, size=3)
    out = dict(U=U, S=S, V=V, lut_w=lut_w,
               g_xy=rng.uniform(0, 1, size=(K, d.Dsy, d.Dsx)),
               g_xc=rng.uniform(0, 1, size=(K, d.Dsx, d.Dsc)),
               g_yc=rng.uniform(0, 1, size=(K, d.Dsy, d.Dsc)),
               grid_w=rng.uniform(-0.05, 0.05, size=(K, 4)))
    return {k: np.ascontiguousarray(v.astype(np.float32)) for k, v in out.items()}


def stack_params(plist: list) -> dict:
    """Stack per-image parameter dicts along a new leading batch axis."""
    return {k: np.ascontiguousarray(np.stack([p[k] for p in plist])) for k in PARAM_NAMES}


def make_batch(seed: int, B: int, H: int, W: int, d: Dims, mode: str = "mix"):
    """B images of one size with their own factors: (x [B][3][H][W], params
    with a leading B axis)."""
    rng = np.random.default_rng(seed)
    xs, ps = [], []
    for _ in range(B):
        xs.append(make_image(rng, H, W, mode=mode))
        ps.append(make_params(rng, d))
    return np.ascontiguousarray(np.stack(xs)), stack_params(ps)


def ragged_sizes(seed: int = SEED_BASE + 2, n: int = 16):
    """n (W, H) sizes drawn uniformly from 480p, 720p, 1080p, 1440p and 4K."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(BATCH_SIZES), size=n)
    return [BATCH_SIZES[i] for i in idx]


def make_ragged(seed: int = SEED_BASE + 2, n: int = 16, sizes=None, mode: str = "mix"):
    """Ragged batch: list of (x [3][H][W], Dims, params) with per-image seeds."""
    sizes = sizes if sizes is not None else ragged_sizes(seed, n)
    out = []
    for j, (W, H) in enumerate(sizes):
        rng = np.random.default_rng(image_seed(j) + seed)
        d = spatial_dims(H, W)
        out.append((make_image(rng, H, W, mode=mode), d, make_params(rng, d)))
    return out


def make_upstream(seed: int, shape) -> np.ndarray:
    """Random float32 upstream gradient ~ N(0,1)."""
    return np.random.default_rng(seed).standard_normal(size=shape).astype(np.float32)


# ---------------------------------------------------------------- generator inputs

GEN_M, GEN_HIDDEN = 8, 8
GEN_CH = (3, 8, 16, 32, 64, 64)


def make_lut3d(rng: np.random.Generator, D: int = 33, kind: str = "photo") -> np.ndarray:
    """Synthetic 3D LUT [3 out][D r][D g][D b] on the vertex grid.
    identity: out_c = in_c.  photo: a seeded photo-style grade (per-channel
    gamma, near-identity colour matrix, saturation about the luma, and a
    split-toning term r*g*b that no sum of 2D tables can express), clipped to
    [0,1].  smooth: identity plus a few seeded low-frequency 3D cosines."""
    v = np.linspace(0.0, 1.0, D)
    r, g, b = np.meshgrid(v, v, v, indexing="ij")
    rgb = np.stack([r, g, b])
    if kind == "identity":
        return rgb.copy()
    if kind == "photo":
        gam = rng.uniform(0.8, 1.25, 3)
        x = rgb ** gam[:, None, None, None]
        M = np.eye(3) + rng.uniform(-0.08, 0.08, (3, 3))
        x = np.einsum("cd,dijk->cijk", M, x)
        lum = 0.299 * x[0] + 0.587 * x[1] + 0.114 * x[2]
        x = lum + rng.uniform(0.8, 1.3) * (x - lum)
        x = x + rng.uniform(-0.3, 0.3, 3)[:, None, None, None] * (r * g * b)
        return np.clip(x, 0.0, 1.0)
    if kind == "smooth":
        x = rgb.copy()
        for _ in range(4):
            f = rng.integers(1, 3, 3)
            ph = rng.uniform(0, 2 * np.pi, 3)
            a = rng.uniform(-0.05, 0.05, 3)
            x += a[:, None, None, None] * np.cos(np.pi * (f[0] * r + f[1] * g + f[2] * b) + ph[:, None, None, None])
        return x
    raise ValueError(kind)


def generator_shapes(K: int):
    """(name, shape) of the generator's weights in the flat FP32 layout
    documented with svdlut_generator_forward (include/svdlut.h)."""
    heads = (K * 3 * 17 * 17, K * 4, 9 * (33 * 8 + 8 + 33 * 8), 12)
    out = []
    for i in range(5):
        cin, cout = GEN_CH[i], GEN_CH[i + 1]
        out += [(f"conv{i}.w", (cout, cin, 3, 3)), (f"conv{i}.b", (cout,))]
        if i < 4:
            out += [(f"in{i}.g", (cout,)), (f"in{i}.b", (cout,))]
    for h, n in zip(("s", "sw", "t", "tw"), heads):
        out += [(f"h{h}.w1", (GEN_HIDDEN, 32 * GEN_M)), (f"h{h}.b1", (GEN_HIDDEN,)),
                (f"h{h}.w2", (n, GEN_HIDDEN)), (f"h{h}.b2", (n,))]
    return out


def generator_init(K: int, rng: np.random.Generator, final_scale: float = 0.0) -> np.ndarray:
    """Seeded initial weights (float64 flat blob).  Convolutions and first FC
    layers: zero-mean normal with variance 2/fan_in resp. 1/fan_in; biases 0;
    InstanceNorm scale 1, shift 0.  The last FC layer of every head: N(0,
    final_scale) (zero when final_scale = 0), its bias the identity factors
    (all grid terms off), so that at final_scale = 0 the predicted transform
    is the identity for every image."""
    parts = {}
    for n, s in generator_shapes(K):
        if n.startswith("conv") and n.endswith(".w"):
            parts[n] = rng.normal(0.0, np.sqrt(2.0 / (s[1] * 9)), size=s)
        elif n.startswith("in") and n.endswith(".g"):
            parts[n] = np.ones(s)
        elif n.endswith(".w1"):
            parts[n] = rng.normal(0.0, np.sqrt(1.0 / s[1]), size=s)
        elif n.endswith(".w2"):
            parts[n] = rng.normal(0.0, final_scale, size=s) if final_scale > 0 else np.zeros(s)
        else:
            parts[n] = np.zeros(s)
    ident = identity_params(Dims(33, 8, K, 17, 17, 17))
    parts["ht.b2"] = np.concatenate([ident["U"].ravel(), ident["S"].ravel(), ident["V"].ravel()])
    parts["htw.b2"] = ident["lut_w"].ravel()
    return np.concatenate([parts[n].ravel() for n, _ in generator_shapes(K)])


def torch_photos(gen, B: int, H: int, W: int, device="cuda"):
    """B photo-like synthetic images [B,3,H,W] float32 on `device` from the
    seeded torch.Generator `gen`: per-channel linear ramps plus two seeded
    sinusoids (the smooth tiles of make_image), then a global exposure gain
    U(0.5, 1.5), a per-channel colour cast U(0.75, 1.25), a gamma
    U(0.7, 1.4) and mild pixel noise N(0, 0.01), clipped to [0,1]."""
    import torch
    kw = dict(device=device, generator=gen)
    yy = torch.linspace(0, 1, H, device=device).view(1, 1, H, 1)
    xx = torch.linspace(0, 1, W, device=device).view(1, 1, 1, W)
    u = lambda *s, lo=0.0, hi=1.0: lo + (hi - lo) * torch.rand(*s, **kw)
    img = u(B, 3, 1, 1, lo=0.1, hi=0.5) + u(B, 3, 1, 1, lo=-0.4, hi=0.4) * xx + u(B, 3, 1, 1, lo=-0.4, hi=0.4) * yy
    for _ in range(2):
        amp, fx, fy = u(B, 3, 1, 1, lo=0.05, hi=0.25), u(B, 3, 1, 1, lo=0.5, hi=3.0), u(B, 3, 1, 1, lo=0.5, hi=3.0)
        ph = u(B, 3, 1, 1, hi=2 * np.pi)
        img = img + amp * torch.sin(2 * np.pi * (fx * xx + fy * yy) + ph)
    img = img.clamp(0, 1) * u(B, 1, 1, 1, lo=0.5, hi=1.5) * u(B, 3, 1, 1, lo=0.75, hi=1.25)
    img = img.clamp(1e-6, 1) ** u(B, 1, 1, 1, lo=0.7, hi=1.4)
    img = img + 0.01 * torch.randn(B, 3, H, W, **kw)
    return img.clamp(0, 1).contiguous()
