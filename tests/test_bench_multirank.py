"""The multi-rank path of bench.py on the CPU: two gloo ranks, as torchrun
starts them (one process per rank, rendezvous on 127.0.0.1).  Each rank
times its own replica; the job time is the slowest rank's, and the job
throughput counts every rank's cells.  The reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 * (rank + 1)  # ms this rank took
        job = bench._max_over_ranks(mine)
        mlups = bench._job_mlups(world, 1000, 50, job * 1e-3)
        r, w, loc = bench._dist()
        dist.barrier()
        out.put((rank, mine, job, mlups, (r, w, loc)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_replica():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, job, mlups, env in res:
        assert env == (rank, world, rank)
        assert job == 20.0                      # the slowest rank's 20 ms
        assert mlups == pytest.approx(world * 1000 * 50 / 0.020 / 1e6)


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5) == 3.5
    assert bench._job_mlups(1, 4, 5, 2.0) == pytest.approx(1e-5)
