"""The multi-rank path of bench.py on CPU: world-size-2 gloo ranks (replicas, weak scaling).

bench.py runs one independent replica per GPU; ranks meet only in a barrier and one max-reduce
of their timings, and rank 0 prints the line.  These tests drive that host logic with gloo."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r was slower on the device-timed leg when r == 1 and on e2e when r == 0
        total, e2e = bench.max_over_ranks([1.0 + rank, 3.0 - rank], world, "cpu")
        rate = bench.whole_job_rate(20, 5, world, total)
        out[rank] = (total, e2e, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        total, e2e, rate = res[r]
        assert total == 2.0 and e2e == 3.0  # the slowest rank's time on each leg
        assert rate == pytest.approx(20 * 5 * 2 / 2.0)  # units of both ranks / slowest time


def test_single_rank_is_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]
    assert bench.whole_job_rate(20, 10, 1, 0.5) == pytest.approx(400.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, configs = 1, 3, ""

    assert bench.run_reference(A()) is None
