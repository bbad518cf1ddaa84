"""The multi-rank host logic of bench.py on CPU: two gloo ranks, as
torchrun launches them (one process per GPU on a GPU machine). Every rank runs
its own replica of the workload with no data exchange; the job's time is
the slowest rank's and its throughput counts the units of all ranks. The
reference arm runs on rank 0 only; the other ranks return without work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        # rank r took (r + 1) s for the fused steps and 0.5 (r + 1) s forward only
        t, f = bench.max_over_ranks(dist, [1.0 + rank, 0.5 * (1.0 + rank)], "cpu")
        out[rank] = (t, f, bench.job_rate(world, 1000.0, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_units():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, f, rate = res[r]
        assert t == 2.0 and f == 1.0          # the slowest rank on every rank
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))
    assert bench.run_reference(None) is None   # returns before it reads any argument
    assert called == []


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.job_rate(1, 50.0, 2.0) == 25.0
