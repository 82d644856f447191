"""The multi-GPU path of bench.py on CPU: ranks as gloo processes
(world size 2, 127.0.0.1).  Each rank solves its own problem (weak scaling,
no data-path collective); the job's figures are the slowest rank's time and
the sum of the ranks' start-iterations."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, iters = bench.aggregate(10.0 + 5.0 * rank, 1000 + rank, world)
        out[rank] = (ms, iters, bench.rank_seed(7, rank), bench.rank_seed(3, rank, 4096))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_max_time_and_sum_of_iterations():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, iters, seed, bseed = res[r]
        assert ms == 15.0 and iters == 2001.0  # every rank reports the job's figures
        assert seed == 7 + r and bseed == 3 + 4096 * r  # independent problems per rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate(12.5, 42, 1) == (12.5, 42.0)
