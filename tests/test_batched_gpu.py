"""GPU parity of svdlut_apply_batched (ragged batch, one persistent launch per
64 images) against the FP64 oracle and against per-image svdlut_apply, plus
CUDA-graph capture/replay and the native autotuner."""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def sv():
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return svdlut


def ragged(seed, sizes, dims=None):
    out = []
    for j, (W, H) in enumerate(sizes):
        rng = np.random.default_rng(seed + j)
        d = dims[j] if dims else si.spatial_dims(H, W)
        out.append((si.make_image(rng, H, W), d, si.make_params(rng, d)))
    return out


def run_batch(sv, items, u8=False):
    import torch
    xs = [torch.from_numpy(si.to_u8(x) if u8 else x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    ys = sv.apply_batched(xs, ps)
    torch.cuda.synchronize()
    return [y.cpu().numpy() for y in ys]


def test_ragged_small_batch_matches_oracle(sv):
    sizes = [(64, 48), (130, 33), (1, 1), (257, 96), (40, 200), (5, 3)]
    items = ragged(500, sizes)
    ys = run_batch(sv, items)
    for (x, d, p), y in zip(items, ys):
        assert np.abs(y.astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def test_ragged_mixed_dims_match_oracle(sv):
    sizes = [(100, 60), (70, 80), (128, 64)]
    dims = [si.paper_dims(), si.Dims(17, 4, 3, 5, 6, 9), si.Dims(33, 33, 0, 2, 2, 2)]
    items = ragged(510, sizes, dims)
    ys = run_batch(sv, items)
    for (x, d, p), y in zip(items, ys):
        assert np.abs(y.astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def test_batched_equals_per_image_apply(sv):
    import torch
    items = ragged(520, [(320, 240), (200, 130), (64, 64)])
    ys = run_batch(sv, items)
    for (x, d, p), y in zip(items, ys):
        ref = sv.apply(torch.from_numpy(x).cuda(), sv.to_device(p)).cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-6


def test_ragged_u8_within_one_lsb(sv):
    items = ragged(530, [(96, 64), (33, 17), (200, 100)])
    ys = run_batch(sv, items, u8=True)
    for (x, d, p), y in zip(items, ys):
        ref = oracle.quantize_u8(oracle.forward(d, p, oracle.u8_to_unit(si.to_u8(x))))
        assert np.abs(y.astype(int) - ref.astype(int)).max() <= 1


def test_more_than_one_launch_chunk(sv):
    sizes = [(16 + (j % 5) * 7, 9 + (j % 3) * 5) for j in range(70)]  # 70 images > 64 per launch
    items = ragged(540, sizes, [si.Dims(9, 2, 3, 3, 3, 5)] * 70)
    ys = run_batch(sv, items)
    for (x, d, p), y in zip(items, ys):
        assert np.abs(y.astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def test_cuda_graph_capture_and_replay(sv):
    import torch
    items = ragged(550, [(640, 480), (128, 96), (300, 200)])
    xs = [torch.from_numpy(x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    batch = sv.Batch(xs, ps)
    batch.run()  # warm-up outside the capture (first call sets kernel attributes)
    torch.cuda.synchronize()
    for y in batch.outs:
        y.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
    for _ in range(2):
        for y in batch.outs:
            y.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (x, d, p), y in zip(items, batch.outs):
            assert np.abs(y.cpu().numpy().astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def test_autotune_returns_a_working_shape(sv):
    import torch
    items = ragged(560, [(640, 480), (320, 240)])
    xs = [torch.from_numpy(x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    batch = sv.Batch(xs, ps)
    block_px, ms = batch.autotune(reps=2)
    assert block_px > 0 and ms > 0
    batch.run()
    torch.cuda.synchronize()
    for (x, d, p), y in zip(items, batch.outs):
        assert np.abs(y.cpu().numpy().astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL


def test_bad_image_reports_its_index(sv):
    import ctypes
    import torch
    from paper_2508_16121_gb300 import _lib
    items = ragged(570, [(32, 32), (32, 32)])
    xs = [torch.from_numpy(x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    batch = sv.Batch(xs, ps)
    batch.imgs[1].H = 0
    lib = _lib.load()
    st = lib.svdlut_apply_batched(batch.imgs, 2, 0, None, ctypes.c_void_p(batch.ws.data_ptr()), batch.ws.numel(),
                                  None)
    assert st == _lib.ERR_INVALID_ARG and b"image 1" in lib.svdlut_last_error()


@pytest.mark.slow
def test_sixteen_ragged_images_benchmark_workload(sv):
    """the benchmarked ragged batch (16 images, 480p..4K), sampled against
    the oracle on three images and against per-image apply on all"""
    import torch
    items = si.make_ragged()
    ys = run_batch(sv, items)
    for j in (0, 7, 15):
        x, d, p = items[j]
        assert np.abs(ys[j].astype(np.float64) - oracle.forward(d, p, x)).max() <= TOL
    for (x, d, p), y in zip(items, ys):
        ref = sv.apply(torch.from_numpy(x).cuda(), sv.to_device(p)).cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-6


def test_autotune_cache_round_trip(sv, tmp_path):
    """A tuned launch shape is stored under (GPU, dtype, sizes) and reused
    without timing; the output is unchanged."""
    import torch
    items = si.make_ragged(seed=77, n=3, sizes=((640, 480), (1280, 720), (640, 480)))
    xs = [torch.from_numpy(x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    cache = str(tmp_path / "tune.json")
    b1 = sv.Batch(xs, ps)
    px1, ms1 = b1.autotune(reps=2, cache=cache)
    assert ms1 is not None
    y1 = [y.clone() for y in b1.run()]
    b2 = sv.Batch(xs, ps)
    px2, ms2 = b2.autotune(reps=2, cache=cache)
    assert ms2 is None and px2 == px1 and b2.cfg.schedule == b1.cfg.schedule
    torch.cuda.synchronize()
    for a, b in zip(y1, b2.run()):
        assert torch.equal(a, b)


@pytest.mark.parametrize("block_rows", [16, 128, 0])
def test_both_schedules_give_identical_output(sv, block_rows):
    """Blocks taken from the atomic queue or as contiguous ranges per CTA:
    the same blocks with the same per-pixel arithmetic, so every bit agrees."""
    import torch
    from paper_2508_16121_gb300 import _lib
    items = si.make_ragged(seed=78, n=5, sizes=((640, 480), (1280, 720), (320, 200), (640, 480), (96, 64)))
    xs = [torch.from_numpy(x).cuda() for x, _, _ in items]
    ps = [sv.to_device(p) for _, _, p in items]
    outs = []
    for sched in (_lib.SCHED_QUEUE, _lib.SCHED_RANGES):
        b = sv.Batch(xs, ps)
        b.cfg = _lib.LaunchCfg(block_rows * 128, 0, sched)
        outs.append([y.clone() for y in b.run()])
    torch.cuda.synchronize()
    for a, c in zip(*outs):
        assert torch.equal(a, c)
    for (x, d, p), y in zip(items, outs[1]):
        ref = sv.apply(torch.from_numpy(x).cuda(), sv.to_device(p))
        assert (y - ref).abs().max().item() <= 1e-6


def test_tables_workspace_gives_identical_output(sv):
    """Per-image tables precomputed into the workspace (prep_kernel) against
    every CTA rebuilding them: identical bits, mixed dims and sizes, F32 and
    u8, more than one launch chunk."""
    import torch
    items = si.make_ragged(seed=23, sizes=[(130, 37), (257, 67), (64, 64), (1, 1), (515, 300)] * 14)
    for u8 in (False, True):
        xs = [torch.from_numpy(si.to_u8(x) if u8 else x).cuda() for x, _, _ in items]
        ps = [sv.to_device(p) for _, _, p in items]
        a = [y.clone() for y in sv.Batch(xs, ps, tables=True).run()]
        b = sv.Batch(xs, ps, tables=False).run()
        torch.cuda.synchronize()
        for ya, yb in zip(a, b):
            assert torch.equal(ya, yb)
