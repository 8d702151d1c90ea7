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
