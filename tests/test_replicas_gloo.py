"""The N > 1 path is independent replicas (no data-path collective): the bench reports the units
all ranks processed over the slowest rank's timed region.  Checked with world_size-2 gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, units, ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        tot, ms_max = bench.job_throughput(units[rank], ms[rank], world, device="cpu")
        dist.barrier()
        q.put((rank, tot, ms_max))
    finally:
        dist.destroy_process_group()


def test_job_throughput_sums_units_and_takes_the_slowest_rank():
    world, port = 2, _free_port()
    units, ms = [3, 5], [1000.0, 2000.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, units, ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, tot, ms_max in got:
        assert tot == 8.0 and ms_max == 2000.0
    # whole-job rate: 8 solves in 2 s
    assert got[0][1] / (got[0][2] / 1e3) == pytest.approx(4.0)


def test_single_rank_is_local():
    import bench
    assert bench.job_throughput(7, 12.5, 1) == (7, 12.5)
