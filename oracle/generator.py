"""FP64 CPU oracle of the SVDLUT factor generator -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this module.  Plain numpy, float64.

Architecture (Supp. Sec. A, Tables 8-12; m = 8, M_s = M_sw = M_t = M_tw = 8):
  bilinear downsample of the input to 3 x 256 x 256           (Table 8, row 1)
  5 x [Conv3x3 stride 2 pad 1 -> LeakyReLU -> InstanceNorm]   (Table 8; no IN
      after the 5th), channels 3 -> 8 -> 16 -> 32 -> 64 -> 64
  Dropout(0.5) (training), average pooling 8x8 -> 2x2, reshape to 256 = 32m
  four heads, each FC 256 -> 8 then FC 8 -> n_out (Tables 9-12):
     H_s  -> K*3*Ds^2 2D bilateral grids (planes xy, xc, yc per grid)
     H_sw -> K*(3+1)  grid weights and bias
     H_t  -> 9*(Dt*Ns + Ns + Dt*Ns): U, S, V of the nine 2D LUTs
     H_tw -> 3*(3+1)  LUT weights and bias
Readings (the paper leaves them open; listed in the design notes): LeakyReLU
slope 0.2; InstanceNorm eps 1e-5 with affine scale/shift and biased variance;
bilinear downsample with half-pixel centres (align_corners = False) and no
antialiasing; average pool of 4x4 windows; no nonlinearity between the two FC
layers of a head (a rank-8 factorisation); H_t's output is split as U, then S,
then V, each in [c][pair] order; H_s's as [K][plane xy, xc, yc][17][17].
The parameter count at K = 6 is 160,478, Table 6 ("Ours", 160.478K).

Parity status: the paper prints no activations or outputs of the generator.
Pinned (tests/test_oracle_generator.py): the parameter count (Table 6 and its
ablation rows) of param_layout; conv against brute force on tiny inputs;
downsample, inorm and avgpool4 against their defining invariants;
splitmix64 against the published SplitMix64 outputs; backward against
central differences of forward; in forward, InstanceNorm as the last step of
layers 0-3 (each plane leaves with mean beta_c and variance at most
gamma_c^2) and dropout on the 8x8 features before the pool (one dropped
element moves one pooled feature by -2a/16).  "Parity unpinned", function by
function, because every pin above still passes if the reading is changed:
  forward          the slope 0.2 and eps 1e-5;
  heads_to_params  the split of each head's output (U, S, V order and the
  params_to_heads  [c][pair] / [K][plane] layouts: a swapped U and V block
                   would pass);
  avgpool4         the 4x4 window (8x8 -> 2x2) as the paper's AvgPool;
  downsample       half-pixel centres without antialiasing;
  dropout_mask     keeping an element when the top bit of its SplitMix64
                   output is 0 (the generator itself is pinned).
"""
from __future__ import annotations

import numpy as np

M = 8                  # backbone width m
CH = (3, M, 2 * M, 4 * M, 8 * M, 8 * M)
THUMB = 256
SLOPE = 0.2
EPS = 1e-5
DT, NS, DS = 33, 8, 17  # LUT vertices, SVD rank, grid vertices
HIDDEN = 8


def head_sizes(K: int):
    """output sizes of H_s, H_sw, H_t, H_tw"""
    return (K * 3 * DS * DS, K * 4, 9 * (DT * NS + NS + DT * NS), 12)


def param_layout(K: int):
    """(name, shape) of every parameter, in the flat blob order"""
    out = []
    for i in range(5):
        cin, cout = CH[i], CH[i + 1]
        out += [(f"conv{i}.w", (cout, cin, 3, 3)), (f"conv{i}.b", (cout,))]
        if i < 4:
            out += [(f"in{i}.g", (cout,)), (f"in{i}.b", (cout,))]
    for h, n in zip(("s", "sw", "t", "tw"), head_sizes(K)):
        out += [(f"h{h}.w1", (HIDDEN, 32 * M)), (f"h{h}.b1", (HIDDEN,)),
                (f"h{h}.w2", (n, HIDDEN)), (f"h{h}.b2", (n,))]
    return out


def param_count(K: int) -> int:
    return int(sum(np.prod(s) for _, s in param_layout(K)))


def unpack(blob, K):
    blob = np.asarray(blob, dtype=np.float64)
    p, o = {}, 0
    for n, s in param_layout(K):
        c = int(np.prod(s))
        p[n] = blob[o:o + c].reshape(s)
        o += c
    assert o == blob.size
    return p


def pack(p, K):
    return np.concatenate([np.asarray(p[n], dtype=np.float64).ravel() for n, _ in param_layout(K)])


# ---------------------------------------------------------------- layers

def downsample(x, S=THUMB):
    """[B,3,H,W] -> [B,3,S,S]; output i samples source (i + 1/2) H/S - 1/2,
    clamped to the image, bilinear between the two nearest pixels per axis."""
    B, C, H, W = x.shape

    def axis(n):
        src = (np.arange(S) + 0.5) * (n / S) - 0.5
        src = np.clip(src, 0.0, n - 1)
        i0 = np.floor(src).astype(int)
        i1 = np.minimum(i0 + 1, n - 1)
        return i0, i1, src - i0

    y0, y1, fy = axis(H)
    x0, x1, fx = axis(W)
    top = x[:, :, y0][:, :, :, x0] * (1 - fx) + x[:, :, y0][:, :, :, x1] * fx
    bot = x[:, :, y1][:, :, :, x0] * (1 - fx) + x[:, :, y1][:, :, :, x1] * fx
    return top * (1 - fy)[:, None] + bot * fy[:, None]


def im2col(x):
    """[B,C,H,W] -> patches [B, Ho, Wo, C, 3, 3] of the stride-2 pad-1 3x3 conv"""
    B, C, H, W = x.shape
    Ho, Wo = H // 2, W // 2
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    cols = np.empty((B, Ho, Wo, C, 3, 3))
    for ky in range(3):
        for kx in range(3):
            cols[..., ky, kx] = xp[:, :, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2].transpose(0, 2, 3, 1)
    return cols


def conv(x, w, b):
    """3x3, stride 2, padding 1: out[b,o,i,j] = b[o] + sum_{c,ky,kx} w[o,c,ky,kx] x[b,c,2i-1+ky,2j-1+kx]"""
    cols = im2col(x)
    out = np.tensordot(cols, w, axes=([3, 4, 5], [1, 2, 3]))  # [B,Ho,Wo,Cout]
    return out.transpose(0, 3, 1, 2) + b[None, :, None, None]


def conv_backward(x, w, dout):
    cols = im2col(x)
    dw = np.tensordot(dout.transpose(1, 0, 2, 3), cols, axes=([1, 2, 3], [0, 1, 2]))
    db = dout.sum(axis=(0, 2, 3))
    dcols = np.tensordot(dout.transpose(0, 2, 3, 1), w, axes=([3], [0]))  # [B,Ho,Wo,C,3,3]
    B, C, H, W = x.shape
    Ho, Wo = H // 2, W // 2
    dxp = np.zeros((B, C, H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dxp[:, :, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2] += dcols[..., ky, kx].transpose(0, 3, 1, 2)
    return dxp[:, :, 1:-1, 1:-1], dw, db


def bf16_round(a):
    """Round to bfloat16 (1 sign, 8 exponent, 7 stored mantissa bits), nearest
    even, returned as float64.  Used only to take the LeakyReLU sign decisions
    in the precision the GPU convolution multiplies in."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def lrelu(z):
    return np.where(z > 0, z, SLOPE * z)


def inorm(a, g, b):
    mu = a.mean(axis=(2, 3), keepdims=True)
    var = a.var(axis=(2, 3), keepdims=True)
    xh = (a - mu) / np.sqrt(var + EPS)
    return xh * g[None, :, None, None] + b[None, :, None, None], (xh, var)


def inorm_backward(dy, g, cache):
    xh, var = cache
    n = xh.shape[2] * xh.shape[3]
    dg = (dy * xh).sum(axis=(0, 2, 3))
    db = dy.sum(axis=(0, 2, 3))
    dxh = dy * g[None, :, None, None]
    da = (dxh - dxh.mean(axis=(2, 3), keepdims=True)
          - xh * (dxh * xh).mean(axis=(2, 3), keepdims=True)) / np.sqrt(var + EPS)
    assert n > 0
    return da, dg, db


def avgpool4(a):
    B, C, H, W = a.shape
    return a.reshape(B, C, H // 4, 4, W // 4, 4).mean(axis=(3, 5))


# ---------------------------------------------------------------- model

def heads_to_params(outs, K):
    """split the four head outputs [B, n] into svdlut parameter arrays"""
    hs, hsw, ht, htw = outs
    B = hs.shape[0]
    g = hs.reshape(B, K, 3, DS, DS)
    nu = 9 * DT * NS
    return dict(U=ht[:, :nu].reshape(B, 3, 3, DT, NS), S=ht[:, nu:nu + 9 * NS].reshape(B, 3, 3, NS),
                V=ht[:, nu + 9 * NS:].reshape(B, 3, 3, DT, NS), lut_w=htw.reshape(B, 3, 4),
                g_xy=np.ascontiguousarray(g[:, :, 0]), g_xc=np.ascontiguousarray(g[:, :, 1]),
                g_yc=np.ascontiguousarray(g[:, :, 2]), grid_w=hsw.reshape(B, K, 4))


def params_to_heads(d, K):
    """inverse of heads_to_params for gradients"""
    B = d["U"].shape[0]
    g = np.stack([d["g_xy"], d["g_xc"], d["g_yc"]], axis=2).reshape(B, -1)
    ht = np.concatenate([d["U"].reshape(B, -1), d["S"].reshape(B, -1), d["V"].reshape(B, -1)], axis=1)
    return [g, d["grid_w"].reshape(B, -1), ht, d["lut_w"].reshape(B, -1)]


def forward(blob, x, K, drop_mask=None, thumb=None, conv_operands="fp64"):
    """x: [B,3,H,W] in [0,1].  drop_mask: None (inference) or [B,64,8,8] of
    {0, 2} (keep-and-scale mask of Dropout(0.5)).  thumb: optional
    precomputed [B,3,256,256] thumbnail.  conv_operands="bf16" multiplies the
    convolution's inputs and weights rounded to bfloat16 (accumulating in
    float64), the precision of the tensor-core convolution; the backward
    pass always uses the exact activations and weights.  Returns (params
    dict, cache)."""
    p = unpack(blob, K)
    a = downsample(np.asarray(x, dtype=np.float64)) if thumb is None else np.asarray(thumb, dtype=np.float64)
    cache = {"acts": []}
    for i in range(5):
        xin = a
        if conv_operands == "bf16":
            z = conv(bf16_round(xin), bf16_round(p[f"conv{i}.w"]), p[f"conv{i}.b"])
        else:
            z = conv(xin, p[f"conv{i}.w"], p[f"conv{i}.b"])
        r = lrelu(z)
        if i < 4:
            a, nc = inorm(r, p[f"in{i}.g"], p[f"in{i}.b"])
        else:
            a, nc = r, None
        cache["acts"].append((xin, z, nc))
    if drop_mask is not None:
        a = a * drop_mask
    pooled = avgpool4(a)
    rho = pooled.reshape(pooled.shape[0], -1)
    hidden, outs = [], []
    for h in ("s", "sw", "t", "tw"):
        t = rho @ p[f"h{h}.w1"].T + p[f"h{h}.b1"]
        hidden.append(t)
        outs.append(t @ p[f"h{h}.w2"].T + p[f"h{h}.b2"])
    cache.update(rho=rho, hidden=hidden, drop_mask=drop_mask, feat_shape=a.shape)
    return heads_to_params(outs, K), cache


def backward(blob, K, cache, dparams):
    """gradient of sum(dparams * params) w.r.t. the parameter blob"""
    p = unpack(blob, K)
    g = {}
    douts = params_to_heads(dparams, K)
    rho = cache["rho"]
    drho = np.zeros_like(rho)
    for h, do, t in zip(("s", "sw", "t", "tw"), douts, cache["hidden"]):
        g[f"h{h}.w2"] = do.T @ t
        g[f"h{h}.b2"] = do.sum(axis=0)
        dt = do @ p[f"h{h}.w2"]
        g[f"h{h}.w1"] = dt.T @ rho
        g[f"h{h}.b1"] = dt.sum(axis=0)
        drho += dt @ p[f"h{h}.w1"]
    B, C, H, W = cache["feat_shape"]
    da = np.repeat(np.repeat(drho.reshape(B, C, H // 4, W // 4), 4, axis=2), 4, axis=3) / 16.0
    if cache["drop_mask"] is not None:
        da = da * cache["drop_mask"]
    for i in reversed(range(5)):
        xin, z, nc = cache["acts"][i]
        if i < 4:
            dr, g[f"in{i}.g"], g[f"in{i}.b"] = inorm_backward(da, p[f"in{i}.g"], nc)
        else:
            dr = da
        dz = dr * np.where(z > 0, 1.0, SLOPE)
        da, g[f"conv{i}.w"], g[f"conv{i}.b"] = conv_backward(xin, p[f"conv{i}.w"], dz)
    return pack(g, K)


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea, Flood 2014; constants as published
    with Java's SplittableRandom): uint64 -> uint64."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def dropout_mask(seed, B, shape=(64, 8, 8)):
    """Dropout(0.5) keep-and-scale mask drawn from a counter-based generator:
    element e (flat index over [B][64][8][8]) is kept (value 2) when the top
    bit of splitmix64(seed * 2^32 + e) is 0, else dropped (value 0)."""
    n = B * int(np.prod(shape))
    idx = (np.uint64(seed) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    keep = (splitmix64(idx) >> np.uint64(63)) == 0
    return (keep * 2.0).reshape((B,) + tuple(shape))


def identity_blob(K, rng=None, scale=0.0):
    """The seeded initial weights of svdlut_inputs.generator_init (identity
    transform at scale = 0, final FC weights N(0, scale) otherwise)."""
    import svdlut_inputs as si
    rng = rng if rng is not None else np.random.default_rng(0)
    blob = si.generator_init(K, rng, scale)
    assert blob.size == param_count(K)
    return blob
