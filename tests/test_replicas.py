"""The multi-GPU path is replicas only (each rank factors its own matrix, no data-path
collective): bench.py's rank plumbing -- process-group setup, barriers, the maximum of the
per-rank times and the whole-job rate -- checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup("gloo")
    bench.barrier(w)
    ms = 10.0 + 5.0 * r                       # the second rank is the slower one
    ms_max = bench.max_over_ranks(ms, w, torch.device("cpu"))
    out.put((r, w, ms_max, bench.whole_job_rate(4, w, ms_max)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for _, w, ms_max, rate in res:
        assert w == 2 and ms_max == pytest.approx(15.0)
        assert rate == pytest.approx(2 * 4 / 0.015)   # 8 factorizations in the slowest 15 ms


def test_single_process_rate_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(10, 1, 20.0) == pytest.approx(500.0)
