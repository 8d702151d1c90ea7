"""Host logic of bench.py's multi-rank run on CPU: two gloo ranks on
127.0.0.1 take the barrier, agree on the slowest rank's time and report the
whole-job rate (units of all ranks over that time).  No GPU is touched."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    b = _bench()
    w, r, _ = b.dist_init(backend="gloo")
    b.barrier(w)
    ms = 10.0 + 5.0 * r  # rank 1 is the slow one
    ms_max = b.max_over_ranks(w, ms)
    q.put((r, w, ms_max, b.job_throughput(w, 8.2944, ms_max)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1]
    for _, w, ms_max, rate in out:
        assert w == 2
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 8.2944 / 0.015)


def test_single_rank_defaults():
    b = _bench()
    assert b.max_over_ranks(1, 3.5) == 3.5
    assert b.job_throughput(1, 8.2944, 1.0) == pytest.approx(8294.4)


def test_reference_arm_line_on_cpu():
    """bench.py --impl reference times the FP64 oracle on the host and prints
    one JSON line with the headline's metric and unit, its sample and an e2e
    entry that moves no bytes between host and device."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    j = json.loads(line)
    b = _bench()
    assert j["impl"] == "reference" and j["metric"] == b.METRIC and j["unit"] == "Mpix/s"
    assert j["value"] > 0 and j["higher_is_better"] is True and j["steps"] == 2
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert "rows" in j["cpu_baseline"]["sample"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0


def test_spread_and_profiled_traffic(tmp_path, monkeypatch):
    """Per-step spread (median, p10, p90) and the DRAM counters of the
    headline kernel, read from the JSON beside its ncu summary only when they
    were taken on the current kernel sources."""
    import json
    b = _bench()
    s = b.spread([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0, 10.0, 11.0])
    assert s["median"] == 6.0 and s["p10"] == 2.0 and s["p90"] == 10.0 and s["steps"] == 11
    counters = tmp_path / "c.json"
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "PROFILE_COUNTERS", "c.json")
    monkeypatch.setattr(b, "kernel_hash", lambda read=None: "abc")
    counters.write_text(json.dumps({"kernel_sources_sha256_16": "abc", "dram_bytes_per_launch": 123}))
    assert b.profiled_traffic() == 123
    assert b.profiled_limiter() is None  # no limiter counters recorded
    counters.write_text(json.dumps({"kernel_sources_sha256_16": "abc", "dram_bytes_per_launch": 123,
                                    "lsu_wavefronts_pct_of_peak": 76.0, "shared_wavefronts_per_pixel": 2.86}))
    lim = b.profiled_limiter()
    assert lim["frac"] == 0.76 and lim["shared_wavefronts_per_pixel"] == 2.86
    counters.write_text(json.dumps({"kernel_sources_sha256_16": "old", "dram_bytes_per_launch": 123,
                                    "lsu_wavefronts_pct_of_peak": 76.0}))
    assert b.profiled_traffic() is None and b.profiled_limiter() is None
    counters.write_text("not json")
    assert b.profiled_traffic() is None
