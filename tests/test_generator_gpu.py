"""GPU parity of the learned factor generator (svdlut_generator_* through the
C ABI) against the FP64 generator oracle.

The convolutions run on BF16 tensor cores (FP32 accumulation), so the bar is
relative: every predicted parameter array within 2e-2 of the oracle's (norm
of the difference over the norm of the reference), weight gradients with
cosine similarity >= 0.999 to the FP64 oracle's, and every parameter group
of the gradient within its bound of the FP64 oracle (GRAD_GROUP_BOUNDS:
3 % for the heads, 20 % for the last conv layer and its norm, 50 % for the
early layers).  Those bounds are about twice what the FP64 oracle itself
moves when only its convolution operands are rounded to BF16 (LeakyReLU
decisions near zero, amplified by InstanceNorm's backward); the CPU test
test_oracle_generator.py pins that margin.

A second, tighter gate compares with the oracle run with BF16-rounded
convolution operands (conv_operands="bf16"): the tensor-core kernels round
exactly those operands, so what remains is FP32 accumulation and FP32
normalisation statistics.  Forward parameters: within 1.5e-3 (observed
<= 4e-4 over the cases here); gradient groups: the heads within 5e-3
(observed <= 7e-4), the convolution and norm layers within 0.1 (observed
<= 0.04: LeakyReLU decisions of values within FP32 rounding of zero still
differ).  Dropout masks, Adam and MSE are compared exactly / to FP32
rounding.
"""
import numpy as np
import pytest

import svdlut_inputs as si
from oracle import generator as G
from test_oracle_generator import grad_group_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def make_blob(K, seed):
    rng = np.random.default_rng(seed)
    blob = G.identity_blob(K, rng, scale=0.05)
    return blob + rng.normal(0, 0.01, size=blob.shape) * (np.abs(blob) > 0)


def gpu_gen(sv, K, blob, B=4):
    import torch
    w = torch.from_numpy(blob.astype(np.float32)).cuda()
    return sv.Generator(K, w, max_batch=B)


def rel(a, r):
    return np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)


@pytest.mark.parametrize("K", [6, 8])
def test_param_count(sv, K):
    from paper_2508_16121_gb300 import _lib
    assert _lib.load().svdlut_generator_param_count(K) == G.param_count(K)


@pytest.mark.parametrize("K,HW", [(8, (256, 256)), (6, (300, 517)), (3, (64, 80))])
def test_forward_matches_oracle(sv, K, HW):
    import torch
    blob = make_blob(K, 10 + K)
    x = np.stack([si.make_image(np.random.default_rng(20 + j), *HW) for j in range(3)])
    gen = gpu_gen(sv, K, blob)
    out = gen.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = G.forward(blob, x, K)
    ref_b, _ = G.forward(blob, x, K, conv_operands="bf16")
    for k in ref:
        got = out[k].cpu().numpy().astype(np.float64)
        assert rel(got, ref[k]) <= 2e-2, k
        assert rel(got, ref_b[k]) <= 1.5e-3, (k, rel(got, ref_b[k]))


@pytest.mark.parametrize("B", [1, 40])
def test_forward_batch_paths_match_oracle(sv, B):
    """The convolution paths that depend on the batch: B = 1 splits K in
    every layer but the first and leaves single partial tiles; B = 40 takes
    the fused finish (bias, LeakyReLU and per-tile statistics in the
    tensor-core epilogue) in layers 0-2, the 16- and 32-channel ones."""
    import torch
    K = 6
    blob = make_blob(K, 60 + B)
    x = np.stack([si.make_image(np.random.default_rng(300 + j), 48, 64) for j in range(B)])
    gen = gpu_gen(sv, K, blob, B=B)
    out = gen.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = G.forward(blob, x, K)
    ref_b, _ = G.forward(blob, x, K, conv_operands="bf16")
    for k in ref:
        got = out[k].cpu().numpy().astype(np.float64)
        assert rel(got, ref[k]) <= 2e-2, k
        assert rel(got, ref_b[k]) <= 1.5e-3, (k, rel(got, ref_b[k]))


def test_training_dropout_mask_matches_counter_generator(sv):
    import torch
    K, seed = 4, 12345
    blob = make_blob(K, 30)
    x = np.stack([si.make_image(np.random.default_rng(40 + j), 128, 128) for j in range(2)])
    gen = gpu_gen(sv, K, blob)
    out = gen.forward(torch.from_numpy(x).cuda(), training=True, seed=seed)
    torch.cuda.synchronize()
    ref, _ = G.forward(blob, x, K, drop_mask=G.dropout_mask(seed, 2))
    ref_nodrop, _ = G.forward(blob, x, K)
    for k in ("U", "g_xy"):
        got = out[k].cpu().numpy().astype(np.float64)
        assert rel(got, ref[k]) <= 2e-2, k
    # the mask matters: the dropped-out prediction differs from inference
    assert rel(ref["U"], ref_nodrop["U"]) > 1e-3


@pytest.mark.parametrize("training,B,HW", [(False, 3, (200, 240)), (True, 3, (200, 240)), (True, 40, (48, 64))])
def test_backward_matches_oracle(sv, training, B, HW):
    """B = 40: the weight-gradient chunks and input-gradient tiles of a large
    batch, after a forward through the fused finish."""
    import torch
    K, seed = 6, 777
    blob = make_blob(K, 50)
    x = np.stack([si.make_image(np.random.default_rng(60 + j), *HW) for j in range(B)])
    gen = gpu_gen(sv, K, blob, B=B)
    out = gen.forward(torch.from_numpy(x).cuda(), training=training, seed=seed)
    rng = np.random.default_rng(70)
    dparams = {k: rng.normal(size=tuple(v.shape)).astype(np.float32) for k, v in out.items()}
    dw = gen.backward({k: torch.from_numpy(v).cuda() for k, v in dparams.items()})
    torch.cuda.synchronize()
    mask = G.dropout_mask(seed, B) if training else None
    d64 = {k: v.astype(np.float64) for k, v in dparams.items()}
    _, cache = G.forward(blob, x, K, drop_mask=mask)
    ref64 = G.backward(blob, K, cache, d64)
    got = dw.cpu().numpy().astype(np.float64)
    cos = float(got @ ref64) / (np.linalg.norm(got) * np.linalg.norm(ref64))
    assert cos >= 0.999, cos
    pg, p64 = G.unpack(got, K), G.unpack(ref64, K)
    errs = {n: rel(pg[n], p64[n]) for n in p64}
    bad = {n: (e, grad_group_bound(n)) for n, e in errs.items() if e > grad_group_bound(n)}
    # the tighter gate: the oracle with BF16-rounded convolution operands
    _, cache_b = G.forward(blob, x, K, drop_mask=mask, conv_operands="bf16")
    pb = G.unpack(G.backward(blob, K, cache_b, d64), K)
    errs_b = {n: rel(pg[n], pb[n]) for n in p64}
    print("per-group rel. error vs FP64 oracle / vs BF16-operand oracle:",
          {n: (round(errs[n], 4), round(errs_b[n], 4)) for n in p64})
    assert not bad, (bad, errs)
    bad_b = {n: e for n, e in errs_b.items() if e > (5e-3 if n.startswith("h") else 0.1)}
    assert not bad_b, bad_b


def test_backward_is_deterministic(sv):
    import torch
    K = 8
    blob = make_blob(K, 80)
    x = torch.from_numpy(np.stack([si.make_image(np.random.default_rng(90), 128, 128)] * 2)).cuda()
    gen = gpu_gen(sv, K, blob, B=2)
    out = gen.forward(x, training=True, seed=3)
    d = {k: torch.ones_like(v) for k, v in out.items()}
    a = gen.backward(d).cpu().numpy()
    gen.forward(x, training=True, seed=3)
    b = gen.backward(d).cpu().numpy()
    assert np.array_equal(a, b)


def test_adam_and_mse(sv):
    import torch
    rng = np.random.default_rng(100)
    n = 1000
    w, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = np.zeros(n, np.float32), np.zeros(n, np.float32)
    wt, gt, mt, vt = (torch.from_numpy(a.copy()).cuda() for a in (w, g, m, v))
    for step in (1, 2):
        sv.adam_step(wt, gt, mt, vt, step, lr=1e-3)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        w = w - 1e-3 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    assert np.abs(wt.cpu().numpy() - w).max() <= 1e-6
    y, t = rng.uniform(size=5000).astype(np.float32), rng.uniform(size=5000).astype(np.float32)
    dy = torch.empty(5000, device="cuda")
    loss = sv.mse(torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), dy)
    assert abs(float(loss) - np.mean((y.astype(np.float64) - t) ** 2)) <= 1e-6
    assert np.abs(dy.cpu().numpy() - 2 * (y - t) / 5000).max() <= 1e-9


def test_forward_on_4k_frames_matches_oracle(sv):
    """The inference workload's input size: 2 x 3840x2160 frames, bilinear
    downsample to the 256x256 thumbnail included."""
    import torch
    K = 8
    blob = make_blob(K, 120)
    x = np.stack([si.make_image(np.random.default_rng(130 + j), 2160, 3840) for j in range(2)])
    gen = gpu_gen(sv, K, blob, B=2)
    out = gen.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = G.forward(blob, x, K)
    ref_b, _ = G.forward(blob, x, K, conv_operands="bf16")
    for k in ref:
        got = out[k].cpu().numpy().astype(np.float64)
        assert rel(got, ref[k]) <= 2e-2, k
        assert rel(got, ref_b[k]) <= 1.5e-3, (k, rel(got, ref_b[k]))


def test_tensor_core_tiles_complete(sv):
    """The convolutions and both gradient GEMMs run on tcgen05 tensor cores
    with bounded waits: after a forward and a backward pass no tile reported
    an expired wait, and every output is finite."""
    import ctypes
    import torch
    from paper_2508_16121_gb300 import _lib
    lib = _lib.load()
    cnt = ctypes.c_uint32(0)
    assert lib.svdlut_tensor_core_timeouts(ctypes.byref(cnt)) == 0
    K = 6
    blob = make_blob(K, 140)
    x = torch.from_numpy(np.stack([si.make_image(np.random.default_rng(150 + j), 96, 128) for j in range(2)])).cuda()
    gen = gpu_gen(sv, K, blob, B=2)
    out = gen.forward(x, training=True, seed=5)
    assert all(bool(torch.isfinite(v).all()) for v in out.values())
    dw = gen.backward({k: torch.ones_like(v) for k, v in out.items()})
    assert torch.isfinite(dw).all()
    assert lib.svdlut_tensor_core_timeouts(ctypes.byref(cnt)) == 0
    assert cnt.value == 0
