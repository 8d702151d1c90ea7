"""Benchmark of the SVDLUT fused apply on GB300.

Default workload: one 3840x2160 RGB FP32 image per step through svdlut_apply
(fused 2D slicing + 2D LUT transform, D_t=33, rank 8, K=8 spatial grids at
1/8 resolution).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference there is:
the paper ships no code) on the same workload, on the host cores.
Under torchrun (N > 1) each rank runs its own replica on its own GPU
(weak scaling, no collective on the data path); value = all ranks' pixels /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import svdlut_inputs as si  # noqa: E402

H4K, W4K = 2160, 3840
METRIC = "Mpix/s and % HBM peak, SVDLUT apply at 4K (plain vs batched/learned), 1 GB300"
N_SETS = 4  # rotating input/output sets: 4 x 199 MB > 129 MB L2


KERNEL_SOURCES = ("paper_2508_16121_gb300/csrc/apply_kernel.cuh", "paper_2508_16121_gb300/csrc/apply_launch.cuh",
                  "paper_2508_16121_gb300/csrc/svdlut_apply.cu")
# ncu counters of the headline kernel (dram bytes per launch), with the hash
# of the kernel sources they were taken on
PROFILE_COUNTERS = "profiles/apply_kernel_f32_3840x2160_mix.json"


def _code_only(src: str) -> str:
    """Source text without comments and blank lines, so that a comment edit
    does not detach the recorded counters from the code they were taken on."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(l.rstrip() for l in src.splitlines() if l.strip())


def kernel_hash(read=None) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def profiled_counters():
    """The committed ncu counters of the headline kernel, if they were taken
    on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, PROFILE_COUNTERS)) as f:
            j = json.load(f)
    except (OSError, ValueError):
        return None
    if not isinstance(j, dict) or j.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    return j


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu counters (None unless
    taken on the current kernel sources)."""
    j = profiled_counters()
    v = j.get("dram_bytes_per_launch") if j else None
    return int(v) if isinstance(v, (int, float)) else None


def profiled_limiter():
    """The resource that bounds the headline kernel, from the same counters:
    shared-memory (LSU) wavefronts as a fraction of their peak."""
    j = profiled_counters()
    v = j.get("lsu_wavefronts_pct_of_peak") if j else None
    if not isinstance(v, (int, float)):
        return None
    return {"resource": "L1 LSU data-pipe wavefronts (shared-memory gathers)", "frac": round(v / 100.0, 3),
            "shared_wavefronts_per_pixel": j.get("shared_wavefronts_per_pixel"),
            "source": "ncu l1tex__data_pipe_lsu_wavefronts, " + PROFILE_COUNTERS}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algo_bytes_apply(H, W, d: si.Dims, io_bytes: int) -> int:
    """Algorithmic bytes of one fused apply: read x and write y (3 planes),
    read the grid planes, grid weights and SVD factors once."""
    px = H * W
    grids = d.K * (d.Dsy * d.Dsx + d.Dsx * d.Dsc + d.Dsy * d.Dsc + 4) * 4
    factors = (2 * 9 * d.D_t * d.rank + 9 * d.rank + 12) * 4
    return px * 3 * io_bytes * 2 + grids + factors


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(backend=None):
    """One process per GPU under torchrun: (world, rank, local).  NCCL on a
    GPU machine; gloo when CUDA is absent (host-logic tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    """Maximum of a per-rank time over all ranks (the job's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, ms_max: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's
    time (weak scaling: every rank runs the same per-rank workload)."""
    return world * units_per_rank / (ms_max / 1e3)


def run_ours(args, world, rank, local):
    import torch
    import paper_2508_16121_gb300 as svdlut
    from paper_2508_16121_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W = H4K, W4K
    d = si.spatial_dims(H, W)
    sets = []
    for s in range(N_SETS):
        x, p = si.make_batch(si.config_seed(1) + 1000 * rank + s, 1, H, W, d)
        sets.append((torch.from_numpy(x).to(dev), svdlut.to_device(p, dev), torch.empty_like(torch.from_numpy(x), device=dev)))
    stream = torch.cuda.current_stream(dev)

    def step(i):
        xt, pt, yt = sets[i % N_SETS]
        svdlut.apply(xt, pt, out=yt)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    # The timed region: K calls back to back, events only at its two ends (an
    # event between two calls would end the overlap of one call's prep_kernel
    # with the previous call's apply_kernel, a programmatic dependent launch).
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for i in range(args.steps):
            step(i)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = max_over_ranks(world, t0.elapsed_time(t1))
    kern_ms = total_ms / args.steps
    clocks = clk.summary()
    # The spread (median, p10, p90) from a second pass of K calls with an
    # event pair around each (which serialises the calls).
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    step_stats = spread([a.elapsed_time(b) for a, b in ev])

    # ---- u8 variant (same frames quantised) ----
    u8_sets = [(torch.from_numpy(si.to_u8(s[0].cpu().numpy())).to(dev), s[1]) for s in sets]
    u8_out = torch.empty_like(u8_sets[0][0])
    for i in range(3):
        svdlut.apply(u8_sets[i % N_SETS][0], u8_sets[i % N_SETS][1], out=u8_out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(args.steps):
        svdlut.apply(u8_sets[i % N_SETS][0], u8_sets[i % N_SETS][1], out=u8_out)
    b.record(stream)
    torch.cuda.synchronize()
    u8_ms = a.elapsed_time(b) / args.steps

    # ---- image regimes (same 4K workload, all-noise / all-smooth pixels) ----
    regimes = {}
    for mode in ("noise", "smooth"):
        xr, pr = si.make_batch(si.config_seed(1) + 7, 1, H, W, d, mode=mode)
        xr_t, pr_t = torch.from_numpy(xr).to(dev), svdlut.to_device(pr, dev)
        yr_t = torch.empty_like(xr_t)
        regimes[mode] = round(H * W / 1e6 / (time_calls(lambda: svdlut.apply(xr_t, pr_t, out=yr_t), args.steps,
                                                         stream) / 1e3), 1)
        del xr_t, yr_t

    # ---- the paper's own transform sizes (K=6 grids of 17^3) on the same 4K image ----
    dp = si.paper_dims()
    xq, pq = si.make_batch(si.config_seed(1) + 11, 1, H, W, dp)
    xq_t, pq_t = torch.from_numpy(xq).to(dev), svdlut.to_device(pq, dev)
    yq_t = torch.empty_like(xq_t)
    paper_ms = time_calls(lambda: svdlut.apply(xq_t, pq_t, out=yq_t), args.steps, stream)
    paper_cfg = {"value": round(H * W / 1e6 / (paper_ms / 1e3), 1), "unit": "Mpix/s", "ms": round(paper_ms, 5),
                 "GB/s": round(algo_bytes_apply(H, W, dp, 4) / (paper_ms / 1e3) / 1e9, 1),
                 "workload": "1x3840x2160 FP32, D_t=33 rank 8, K=6 grids 17x17x17"}
    del xq_t, yq_t

    # ---- the paper's original, unfused structure (maps and fused image through HBM) ----
    original = {}
    for name, dd, (xx, pp_) in (("1/8-res K=8", d, (sets[0][0], sets[0][1])), ("paper K=6 17^3", dp, (None, None))):
        if xx is None:
            xx, pp_ = torch.from_numpy(xq).to(dev), svdlut.to_device(pq, dev)
        frng = np.random.default_rng(si.config_seed(1) + 13)
        Wf = frng.normal(0, 0.15, (3, dd.K + 3))
        Wf[np.arange(3), np.arange(3)] += 1.0
        fus = torch.tensor(np.concatenate([Wf.ravel(), np.zeros(3)]), dtype=torch.float32, device=dev)
        ws_o = torch.empty(svdlut.original_workspace_bytes(pp_, 1, H, W), dtype=torch.uint8, device=dev)
        yo = torch.empty_like(xx)
        t_o = time_calls(lambda: svdlut.apply_original(xx, pp_, fus, out=yo, workspace=ws_o), max(3, args.steps // 4),
                         stream)
        t_f = time_calls(lambda: svdlut.apply(xx, pp_, out=yo), max(3, args.steps // 4), stream)
        bytes_o = H * W * (60 + 8 * dd.K)  # X read twice, K maps written and read, Xbar written and read, Y written
        original[name] = {"original_ms": round(t_o, 4), "fused_ms": round(t_f, 4),
                          "fused_speedup": round(t_o / t_f, 2),
                          "original_GB/s": round(bytes_o / (t_o / 1e3) / 1e9, 1),
                          "original_bytes_per_px": 60 + 8 * dd.K}
        del ws_o, yo

    # ---- 16-bit and interleaved pixel formats on the same 4K frame ----
    io_formats = run_io_variant(svdlut, torch, dev, stream, args, sets[0][0], sets[0][1], d)

    # ---- the 3D LUT of Eq. 3 against its best 2D-LUT fit (Eq. 4) on the same 4K image ----
    lut3d = run_lut3d_variant(svdlut, torch, dev, stream, args, sets[0][0])

    # ---- ragged batch: 16 images 480p..4K, one graph-captured launch vs 16 plain calls ----
    batched = run_batched_variant(svdlut, torch, dev, stream, args)

    # ---- adjoint: 8 x 1920x1080 FP32, all gradients ----
    backward = run_backward_variant(svdlut, torch, dev, stream, args)

    # ---- learned: generator + apply on 4 x 4K in one graph; training step ----
    learned = run_learned_variant(svdlut, torch, dev, stream, args)

    # ---- end to end through the public API with pinned host buffers:
    # svdlut_apply_host reads and writes the pinned host frames in place over
    # the CPU-GPU link; every step moves the whole frame in and out ----
    xh = sets[0][0].cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    pd = sets[0][1]
    for _ in range(3):
        svdlut.apply_host(xh, pd, out=yh)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        svdlut.apply_host(xh, pd, out=yh)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(world, a.elapsed_time(b) / args.steps)
    # the same, with whole-frame copies and svdlut_apply in sequence
    xd, pd, yd = sets[0]
    a.record(stream)
    for _ in range(max(3, args.steps // 4)):
        xd.copy_(xh, non_blocking=True)
        svdlut.apply(xd, pd, out=yd)
        yh.copy_(yd, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_serial_ms = a.elapsed_time(b) / max(3, args.steps // 4)

    mpix = H * W / 1e6
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, mpix, ms_per_step)
    peak, peak_src = peaks()
    bytes_launch = algo_bytes_apply(H, W, d, 4)
    achieved = bytes_launch / (kern_ms / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; 64x64 checkerboard of U(0,1) noise and smooth gradients)",
        "config": {"workload": "plain svdlut_apply, 1x3840x2160 RGB FP32, D_t=33 rank 8, K=8 grids "
                               "480x270x17 (1/8 res)", "global_batch": world, "image": "3840x2160",
                   "parallelism": f"replicas x{world}",
                   "l2": f"rotating {N_SETS} input/output sets ({N_SETS * bytes_launch / 1e6:.0f} MB) > 129 MB L2"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": profiled_traffic(),
                     "limiter": profiled_limiter(),
                     "kernel": "apply_kernel<Io<InF32, OutF32>, 16, false>",
                     "timed": "CUDA events around the K back-to-back calls of the timed region, per call "
                              "(prep_kernel + apply_kernel)",
                     "bytes_per_launch": bytes_launch,
                     "kernel_ms": round(kern_ms, 5),
                     "per_call_events": dict(step_stats, note="second pass, an event pair around each call"),
                     "frac_at_median_per_call_events": round(bytes_launch / (step_stats["median"] / 1e3) / 1e9
                                                             / peak, 4),
                     "peak_source": peak_src,
                     "kernel_sources_sha256_16": kernel_hash()},
        "e2e": {"value": round(job_throughput(world, mpix, e2e_ms), 1), "unit": "Mpix/s",
                "h2d_bytes_per_step": int(xh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * 4),
                "api": "svdlut_apply_host (pinned host frames read and written in place over NVLink-C2C)",
                "serial_copies_Mpix/s": round(mpix / (e2e_serial_ms / 1e3), 1)},
        "gpu_launches": 2 * args.steps,  # prep_kernel + apply_kernel per svdlut_apply_ws call
        "clocks": clocks,
        "variants": {"u8_plain_4k": {"value": round(mpix / (u8_ms / 1e3), 1), "unit": "Mpix/s",
                                     "ms": round(u8_ms, 5),
                                     "GB/s": round(algo_bytes_apply(H, W, d, 1) / (u8_ms / 1e3) / 1e9, 1)},
                     "f32_plain_4k_by_regime_Mpix/s": regimes,
                     "f32_plain_4k_paper_grids": paper_cfg,
                     "original_unfused_structure_4k": original,
                     "io_formats_4k": io_formats,
                     "lut3d_vs_2d_fit_4k": lut3d,
                     "batched_16_ragged": batched,
                     "backward_8x1080p": backward,
                     "learned_4x4k": learned},
    }
    return out, (xh.numpy(), {k: v.cpu().numpy() for k, v in pd.items()}, d)


def spread(ms):
    """median, 10th and 90th percentile of per-step times (ms)"""
    q = np.percentile(np.asarray(ms, dtype=np.float64), [10, 50, 90])
    return {"p10": round(float(q[0]), 5), "median": round(float(q[1]), 5), "p90": round(float(q[2]), 5),
            "steps": len(ms)}


def time_calls(fn, steps, stream, warmup=3):
    """mean ms per call of fn() on `stream`, CUDA events around the loop"""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_io_variant(svdlut, torch, dev, stream, args, x, p, d):
    """svdlut_apply_io on the 4K frame: interleaved 8-bit in and out, and
    16-bit inputs (decoded to FP32 by their own kernel, then the FP32-input
    transform); GB/s counts the call's input and output bytes."""
    H, W = x.shape[-2], x.shape[-1]
    steps = max(3, args.steps // 2)
    grids = algo_bytes_apply(H, W, d, 0)  # the parameter and grid bytes alone
    xh = x.cpu().numpy().reshape(-1, 3, H, W)
    v8 = si.to_u8(xh)
    dv = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
    v16 = np.rint(np.clip(xh, 0.0, 1.0) * 65535.0).astype(np.uint16)
    cases = {"u8_hwc->u8_hwc": (dv(si.to_hwc(v8)), "u8_hwc", "u8_hwc", 6),
             "u16->u8": (dv(v16), "u16", "u8", 9),
             "u16->f32": (dv(v16), "u16", "f32", 18),
             "u16_hwc->u8_hwc": (dv(si.to_hwc(v16)), "u16_hwc", "u8_hwc", 9)}
    out = {}
    for name, (xin, fi, fo, bpp) in cases.items():
        y = svdlut.apply_io(xin, p, fi, fo)
        ms = time_calls(lambda: svdlut.apply_io(xin, p, fi, fo, out=y), steps, stream)
        out[name] = {"value": round(H * W / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s", "ms": round(ms, 5),
                     "GB/s": round((H * W * bpp + grids) / (ms / 1e3) / 1e9, 1), "io_bytes_per_px": bpp}
        del y
    out["workload"] = f"1x{W}x{H}, D_t=33 rank 8, K=8 grids at 1/8 res; inputs = the headline frame quantised"
    out["u16_path"] = "u16_decode_kernel to an FP32 frame (stream-ordered buffer), then the FP32-input apply"
    return out


def run_lut3d_variant(svdlut, torch, dev, stream, args, x):
    """3D LUT transform vs the 2D transform of its least-squares 2D fit, full
    rank and truncated to rank 8 (Eq. 9), for a photo-style and a smooth 33^3
    LUT: speed, fit RMS on the vertex grid and RMS difference on the image."""
    H, W = x.shape[-2], x.shape[-1]
    steps = max(3, args.steps // 4)
    out = {}
    y3, y2 = torch.empty_like(x), torch.empty_like(x)
    for kind in ("photo", "smooth"):
        rng = np.random.default_rng(si.config_seed(1) + 17)
        lut = torch.tensor(si.make_lut3d(rng, 33, kind), dtype=torch.float32, device=dev)[None]
        ws = torch.empty(svdlut._lib.load().svdlut_lut3d_workspace_size(33, 1), dtype=torch.uint8, device=dev)
        t3 = time_calls(lambda: svdlut.lut3d_apply(x, lut, out=y3, workspace=ws), steps, stream)
        tf = time_calls(lambda: svdlut.lut3d_fit2d(lut), steps, stream)
        tables, rms = svdlut.lut3d_fit2d(lut)
        pf = svdlut.fit_params(tables)
        t2 = time_calls(lambda: svdlut.apply(x, pf, out=y2), steps, stream)
        full_rmse = float(torch.sqrt(torch.mean((y2 - y3) ** 2)))
        # rank-8 truncation of each fitted table (host SVD: analysis only)
        u, sv_, vt = np.linalg.svd(tables[0].double().cpu().numpy())
        p8 = dict(pf, U=torch.tensor(u[..., :8], dtype=torch.float32, device=dev)[None].contiguous(),
                  S=torch.tensor(sv_[..., :8], dtype=torch.float32, device=dev)[None].contiguous(),
                  V=torch.tensor(np.swapaxes(vt, -1, -2)[..., :8], dtype=torch.float32, device=dev)[None].contiguous())
        t8 = time_calls(lambda: svdlut.apply(x, p8, out=y2), steps, stream)
        r8_rmse = float(torch.sqrt(torch.mean((y2 - y3) ** 2)))
        out[kind] = {"lut3d_ms": round(t3, 4), "lut3d_Mpix/s": round(H * W / 1e6 / (t3 / 1e3), 1),
                     "lut3d_GB/s": round(H * W * 24 / (t3 / 1e3) / 1e9, 1),
                     "fit2d_ms": round(tf, 4), "fit2d_full_rank_ms": round(t2, 4), "fit2d_rank8_ms": round(t8, 4),
                     "fit_rms_vertex_grid": [round(float(v), 6) for v in rms[0]],
                     "image_rmse_full_rank_vs_3d": round(full_rmse, 6), "image_rmse_rank8_vs_3d": round(r8_rmse, 6)}
    out["workload"] = f"1x{W}x{H} FP32, 33^3 LUTs (seeded photo-style grade and smooth cosine LUT), no grids"
    return out


def run_batched_variant(svdlut, torch, dev, stream, args):
    items = si.make_ragged()
    xs = [torch.from_numpy(x).to(dev) for x, _, _ in items]
    ps = [svdlut.to_device(p, dev) for _, _, p in items]
    batch = svdlut.Batch(xs, ps)
    block_px, _ = batch.autotune(reps=3)
    batch.run()
    torch.cuda.synchronize()
    mpix = sum(x.shape[1] * x.shape[2] for x in xs) / 1e6
    bytes_px = sum(algo_bytes_apply(x.shape[1], x.shape[2], d, 4) for (x, d, _) in items)
    g_b = torch.cuda.CUDAGraph()
    s_cap = torch.cuda.Stream(dev)
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g_b, stream=s_cap):
            batch.run(stream=s_cap)
    ys = [torch.empty_like(x) for x in xs]

    def seq():
        for x, p, y in zip(xs, ps, ys):
            svdlut.apply(x, p, out=y)

    seq()
    torch.cuda.synchronize()
    g_s = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g_s, stream=s_cap):
            for x, p, y in zip(xs, ps, ys):
                svdlut.apply(x, p, out=y, stream=s_cap)
    steps = max(3, args.steps // 4)
    t_b = time_calls(g_b.replay, steps, stream)
    t_s = time_calls(g_s.replay, steps, stream)
    t_e = time_calls(seq, steps, stream)
    return {"images": len(xs), "Mpix": round(mpix, 2), "autotuned_block_px": block_px,
            "autotuned_schedule": "ranges" if batch.cfg.schedule == 1 else "queue",
            "batched_graph": {"value": round(mpix / (t_b / 1e3), 1), "unit": "Mpix/s", "ms": round(t_b, 4),
                              "GB/s": round(bytes_px / (t_b / 1e3) / 1e9, 1)},
            "plain_x16_graph": {"value": round(mpix / (t_s / 1e3), 1), "unit": "Mpix/s", "ms": round(t_s, 4)},
            "plain_x16_eager": {"value": round(mpix / (t_e / 1e3), 1), "unit": "Mpix/s", "ms": round(t_e, 4)},
            "speedup_vs_plain_graph": round(t_s / t_b, 3)}


def run_backward_variant(svdlut, torch, dev, stream, args):
    H, W, B = 1080, 1920, 8
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(3), B, H, W, d)
    xt, pt = torch.from_numpy(x).to(dev), svdlut.to_device(p, dev)
    gt = torch.from_numpy(si.make_upstream(si.config_seed(3) + 1, x.shape)).to(dev)
    ws = torch.empty(1 << 28, dtype=torch.uint8, device=dev)
    steps = max(3, args.steps // 4)
    ms = time_calls(lambda: svdlut.backward(xt, pt, gt, workspace=ws), steps, stream)
    px = B * H * W
    algo = px * 36 + sum(int(v.numel()) * 8 for v in pt.values())  # x, dy in; dx out; params in, grads out
    return {"value": round(px / 1e6 / (ms / 1e3), 1), "unit": "Mpix/s", "ms": round(ms, 4),
            "GB/s": round(algo / (ms / 1e3) / 1e9, 1), "workload": "8 x 1920x1080 FP32, all gradients"}


def run_learned_variant(svdlut, torch, dev, stream, args):
    """Generator (thumbnail, BF16 tensor-core backbone, heads) + one apply
    over 4 x 3840x2160, captured in one CUDA graph, against the plain
    per-image path (4 svdlut_apply calls with given factors)."""
    from paper_2508_16121_gb300 import train
    K, B, H, W = 8, 4, H4K, W4K
    x, _ = si.make_batch(si.config_seed(4), B, H, W, si.Dims(33, 8, K, 17, 17, 17))
    xt = torch.from_numpy(x).to(dev)
    w = torch.tensor(si.generator_init(K, np.random.default_rng(si.config_seed(4)), 0.05), dtype=torch.float32,
                     device=dev)
    gen = svdlut.Generator(K, w, max_batch=B)
    params = gen.forward(xt)
    y = torch.empty_like(xt)
    svdlut.apply(xt, params, out=y)
    torch.cuda.synchronize()
    s_cap = torch.cuda.Stream(dev)
    g_l = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g_l, stream=s_cap):
            gen.forward(xt, out=params, stream=s_cap)
            svdlut.apply(xt, params, out=y, stream=s_cap)
    per = [{k: v[i:i + 1].clone() for k, v in params.items()} for i in range(B)]
    ys = [torch.empty_like(xt[i:i + 1]) for i in range(B)]
    g_p = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g_p, stream=s_cap):
            for i in range(B):
                svdlut.apply(xt[i:i + 1], per[i], out=ys[i], stream=s_cap)
    # Serving throughput: batches back to back, the generator of batch t+1
    # (its own stream, a few SMs) overlapping the transform of batch t (a
    # persistent launch on the other SMs, svdlut_apply_cfg); parameters
    # double-buffered.  The SMs left to the generator come from a short sweep.
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    pp = [gen.empty_params(B) for _ in range(2)]
    ybuf = [torch.empty_like(xt) for _ in range(2)]
    s_gen, s_app = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    e_gen = [torch.cuda.Event() for _ in range(2)]
    e_app = [torch.cuda.Event() for _ in range(2)]
    e_fork, e_join_g, e_join_a = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
    T = 8  # batches per graph replay

    def pipeline(cap_stream, ctas):
        e_fork.record(cap_stream)
        s_gen.wait_event(e_fork)
        s_app.wait_event(e_fork)
        for t in range(T):
            slot = t % 2
            if t >= 2:
                s_gen.wait_event(e_app[slot])  # batch t-2 is done with this parameter buffer
            gen.forward(xt, out=pp[slot], stream=s_gen)
            e_gen[slot].record(s_gen)
            s_app.wait_event(e_gen[slot])
            svdlut.apply(xt, pp[slot], out=ybuf[slot], stream=s_app, ctas=ctas)
            e_app[slot].record(s_app)
        e_join_g.record(s_gen)
        e_join_a.record(s_app)
        cap_stream.wait_event(e_join_g)
        cap_stream.wait_event(e_join_a)

    pipe = None
    for free_sms in (0, 4, 8, 12, 16, 24):
        pipeline(s_cap, n_sm - free_sms)
        torch.cuda.synchronize()
        g_try = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s_cap):
            with torch.cuda.graph(g_try, stream=s_cap):
                pipeline(s_cap, n_sm - free_sms)
        t_try = time_calls(g_try.replay, 3, stream) / T
        if pipe is None or t_try < pipe[1]:
            pipe = (g_try, t_try, free_sms)
    g_pipe, _, free_sms = pipe

    # the plain per-image path as a caller without the generator runs it:
    # factors given on the host, one upload and one svdlut_apply per image
    host = [{k: v[i:i + 1].cpu().pin_memory() for k, v in params.items()} for i in range(B)]
    dev_p = [{k: torch.empty_like(v[i:i + 1]) for k, v in params.items()} for i in range(B)]

    def plain_host():
        for i in range(B):
            for k in host[i]:
                dev_p[i][k].copy_(host[i][k], non_blocking=True)
            svdlut.apply(xt[i:i + 1], dev_p[i], out=ys[i])

    steps = max(3, args.steps // 40)
    t_l = time_calls(g_l.replay, steps, stream)
    t_p = time_calls(g_p.replay, steps, stream)
    t_h = time_calls(plain_host, steps, stream)
    t_pipe = time_calls(g_pipe.replay, max(3, steps // 8), stream) / T
    t_g = time_calls(lambda: gen.forward(xt, out=params), steps, stream)
    mpix = B * H * W / 1e6
    # one training step (batch 64 of 256x256 pairs) through the library kernels
    tr = train.Trainer(K=K, batch=64, size=256, lr=1e-3)
    tr.run(3)
    torch.cuda.synchronize()
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_tr = 20
    a_.record(stream)
    tr.run(n_tr)
    b_.record(stream)
    torch.cuda.synchronize()
    t_tr = a_.elapsed_time(b_) / n_tr
    # the loss terms of that step alone: MSE, then CIE94 added into the same gradient
    xb, ytb = tr.pair(1)
    yb = svdlut.apply(xb, tr.student.forward(xb))
    dyb, ws_l = torch.empty_like(yb), torch.empty(4096, dtype=torch.uint8, device=dev)
    t_mse = time_calls(lambda: svdlut.mse(yb, ytb, dyb, ws=ws_l), steps, stream)
    t_cie = time_calls(lambda: svdlut.cie94(yb, ytb, svdlut.CIE94_WEIGHT, dy=dyb, accumulate=True, ws=ws_l),
                       steps, stream)
    return {"workload": "4 x 3840x2160 FP32, K=8 grids 17^3, D_t=33 rank 8",
            "generator_plus_apply_graph": {"value": round(mpix / (t_l / 1e3), 1), "unit": "Mpix/s",
                                           "ms": round(t_l, 4)},
            "plain_x4_graph": {"value": round(mpix / (t_p / 1e3), 1), "unit": "Mpix/s", "ms": round(t_p, 4),
                               "factors": "device-resident, 4 svdlut_apply in one CUDA graph"},
            "plain_x4_host_factors": {"value": round(mpix / (t_h / 1e3), 1), "unit": "Mpix/s", "ms": round(t_h, 4),
                                      "factors": "pinned host, uploaded per image before each svdlut_apply"},
            "generator_forward_ms": round(t_g, 4),
            "speedup_vs_plain_graph": round(t_p / t_l, 3),
            "speedup_vs_plain_host_factors": round(t_h / t_l, 3),
            "serving_pipelined": {"value": round(mpix / (t_pipe / 1e3), 1), "unit": "Mpix/s",
                                  "ms_per_batch": round(t_pipe, 4),
                                  "how": f"{T} batches per graph; the generator of batch t+1 on its own "
                                         "stream, overlapping the transform of batch t" +
                                         (f" (svdlut_apply_cfg: persistent CTAs on all but {free_sms} SMs)"
                                          if free_sms else " (the transform's CTAs on every SM: the fastest "
                                          "of 0-24 SMs left free)"),
                                  "speedup_vs_plain_graph": round(t_p / t_pipe, 3)},
            "train_step_ms_batch64_256px": round(t_tr, 3),
            "train_loss": "MSE + 0.005 CIE94 (Eq. 11 without LPIPS)",
            "loss_terms_ms_batch64_256px": {"mse_and_grad": round(t_mse, 4), "cie94_and_grad": round(t_cie, 4),
                                            "cie94_Mpix/s": round(64 * 256 * 256 / 1e6 / (t_cie / 1e3), 1)},
            "train_pairs_per_s": round(64 / (t_tr / 1e3), 1)}


def cpu_baseline(x, p, d, reps=2):
    import oracle
    cores = os.cpu_count() or 1
    oracle.forward(d, p, x[..., :64, :], nthreads=cores)  # warm
    t = time.time()
    for _ in range(reps):
        oracle.forward(d, p, x, nthreads=cores)
    dt = time.time() - t
    px = reps * x.shape[-1] * x.shape[-2]
    return {"value": round(px / dt / 1e6, 3), "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} full 3840x2160 FP32 frames through the FP64 oracle, OpenMP over rows "
                      f"({dt:.1f} s wall)"}


def oracle_table(reps_fast=5, reps_slow=3):
    """Timings of the FP64 CPU oracle on the host for the five workloads of
    the benchmark table (Mpix/s, median of repeated runs, one thread and all
    host cores): 256x256 apply, 3840x2160 apply, the 16-image ragged batch
    (sum over its images), the adjoint of 8 x 1920x1080 (the oracle's adjoint
    is single-threaded) and the generator forward per 3840x2160 image."""
    import oracle
    from oracle import generator as G
    oracle.build()
    cores = os.cpu_count() or 1

    def med(fn, reps):
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t)
        return statistics.median(ts)

    out = {"cores": cores, "unit": "Mpix/s (median of repeated runs)"}
    for name, H, W in (("config0_256x256", 256, 256), ("config1_3840x2160", H4K, W4K)):
        d = si.spatial_dims(H, W)
        x, p = si.make_batch(si.config_seed(0 if H == 256 else 1), 1, H, W, d)
        oracle.forward(d, p, x[..., :8, :], nthreads=cores)  # warm
        t1 = med(lambda: oracle.forward(d, p, x, nthreads=1), reps_slow if H > 256 else reps_fast)
        tn = med(lambda: oracle.forward(d, p, x, nthreads=cores), reps_fast)
        out[name] = {"1_core": round(H * W / t1 / 1e6, 3), f"{cores}_cores": round(H * W / tn / 1e6, 3)}
    items = si.make_ragged()
    px = sum(x.shape[1] * x.shape[2] for x, _, _ in items)

    def ragged(n):
        for x, d, p in items:
            oracle.forward(d, p, x, nthreads=n)
    t1, tn = med(lambda: ragged(1), reps_slow), med(lambda: ragged(cores), reps_fast)
    out["config2_16_ragged"] = {"1_core": round(px / t1 / 1e6, 3), f"{cores}_cores": round(px / tn / 1e6, 3),
                                "Mpix": round(px / 1e6, 2)}
    Hb, Wb, B = 1080, 1920, 8
    db = si.spatial_dims(Hb, Wb)
    xb, pb = si.make_batch(si.config_seed(3), B, Hb, Wb, db)
    gb = si.make_upstream(si.config_seed(3) + 1, xb.shape)
    t1 = med(lambda: oracle.backward(db, pb, xb, gb), reps_slow)
    out["config3_backward_8x1080p"] = {"1_core": round(B * Hb * Wb / t1 / 1e6, 3), "s_per_call": round(t1, 2),
                                       "note": "the oracle's adjoint runs on one core"}
    K = 8
    blob = G.identity_blob(K, np.random.default_rng(si.config_seed(4)), scale=0.05)
    x4, _ = si.make_batch(si.config_seed(4), 1, H4K, W4K, si.Dims(33, 8, K, 17, 17, 17))
    tg = med(lambda: G.forward(blob, x4, K), reps_fast)
    out["config4_generator_forward"] = {"ms_per_image": round(tg * 1e3, 2),
                                        "note": "numpy FP64 with its default BLAS threads; input 3840x2160"}
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    H, W = H4K, W4K
    d = si.spatial_dims(H, W)
    x, p = si.make_batch(si.config_seed(1), 1, H, W, d)
    x, p = x[0], {k: v[0] for k, v in p.items()}
    cores = os.cpu_count() or 1
    # Each step is a bounded sample of the 4K frame: its first `rows` rows,
    # sized from the warm-up rate so that all steps take about a minute.
    t = time.time()
    for _ in range(max(1, args.warmup)):
        oracle.forward(d, p, x[:, :64], nthreads=cores)
    px_per_s = max(1, args.warmup) * 64 * W / max(time.time() - t, 1e-6)
    rows = int(min(H, max(1, 60.0 * px_per_s / max(args.steps, 1) / W)))
    xs = np.ascontiguousarray(x[:, :rows])
    t = time.time()
    for _ in range(args.steps):
        oracle.forward(d, p, xs, nthreads=cores)
    dt = time.time() - t
    ms = dt * 1e3 / args.steps
    v = rows * W / 1e6 / (ms / 1e3)
    sample = (f"{args.steps} steps, each the first {rows} of 2160 rows of the 3840x2160 frame "
              f"({rows * W / 1e6:.2f} Mpx) through the FP64 CPU oracle")
    return {
        "metric": METRIC, "value": round(v, 3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
        "config": {"workload": "plain svdlut_apply, 1x3840x2160 RGB FP32, D_t=33 rank 8, K=8 grids "
                               "480x270x17 (1/8 res)", "global_batch": 1, "image": "3840x2160",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": round(v, 3), "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the FP64 CPU oracle on the five benchmark workloads and print one JSON line")
    args = ap.parse_args()
    if args.oracle_table:
        print(json.dumps(oracle_table()), flush=True)
        return
    args.warmup = max(3, args.warmup)
    world, rank, local = (1, 0, 0)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        if args.impl == "reference":
            rank = int(os.environ.get("RANK", "0"))
            if rank != 0:
                return
            world = int(os.environ.get("WORLD_SIZE", "1"))
        else:
            world, rank, local = dist_init()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out, sample = run_ours(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            x, p, d = sample
            out["cpu_baseline"] = cpu_baseline(x, p, d)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
