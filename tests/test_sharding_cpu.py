"""The multi-rank (weak scaling) host logic on CPU: two gloo ranks on 127.0.0.1.

Each rank estimates its own fields; no data moves between ranks; the job rate
is the units all ranks processed over the slowest rank's time.  A rank that
fails must not leave the others hanging in a collective.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1904_11055_gb300 import sharding  # noqa: E402


def test_unit_ranges_partition_the_units():
    for n in (0, 1, 7, 512, 1000):
        for world in (1, 2, 3, 8):
            parts = [sharding.unit_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, _) in zip(parts, parts[1:]):
                assert b == c
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.unit_range(4, 2, 2)


def test_single_rank_reduces_to_plain_arithmetic():
    assert not dist.is_initialized()
    assert sharding.max_over_ranks(2.5) == 2.5
    assert sharding.job_rate(10, 2.0) == 5.0
    assert sharding.field_seed(2, 0) == 2 and sharding.field_seed(2, 1) == 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from datetime import timedelta

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=20))
    try:
        r, w, _ = sharding.rank_env()
        assert (r, w) == (rank, world)
        units = [3, 5][rank]
        seconds = [1.0, 2.0][rank]
        a, b = sharding.unit_range(8, world, rank)
        rate = sharding.job_rate(units, seconds)
        tmax = sharding.max_over_ranks(seconds)
        if rank == fail_rank:
            raise RuntimeError("planted failure before the second collective")
        dist.barrier()
        results[rank] = (rate, tmax, a, b, sharding.field_seed(2, rank))
    except RuntimeError as e:
        results[rank] = ("error", str(e)[:80])
    finally:
        dist.destroy_process_group()


def _run(fail_rank):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), results, fail_rank), nprocs=2, join=True,
                           start_method="spawn")
        return dict(results)


def test_two_gloo_ranks_aggregate_as_one_job():
    res = _run(fail_rank=-1)
    assert res[0][:2] == (4.0, 2.0) and res[1][:2] == (4.0, 2.0)  # (3 + 5) units / slowest 2 s
    assert (res[0][2], res[0][3], res[1][2], res[1][3]) == (0, 4, 4, 8)
    assert res[0][4] != res[1][4]


def test_a_failing_rank_ends_the_others_collective_with_an_error():
    res = _run(fail_rank=1)
    assert res[1][0] == "error"
    assert res[0][0] == "error"  # rank 0's barrier ends with an error instead of hanging
