"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank times its own
replica of the step; the job's time is the slowest rank's (all-reduce MAX) and its rate the
units of all ranks over that time.  Rendezvous on 127.0.0.1."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    mine = 1.25 + 0.5 * r                     # this rank's step time, seconds
    t = bench.max_over_ranks(mine, w, torch.device("cpu"))
    rate = bench.job_rate(6 * 5, w, t)
    out.put((r, w, local, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t, rate) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t == pytest.approx(1.75)            # max over ranks
        assert rate == pytest.approx(2 * 30 / 1.75)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_rate(30, 1, 2.0) == 15.0
