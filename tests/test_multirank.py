"""Multi-process path of the benchmark on CPU ranks (gloo, world size 2).

Images are independent, so N GPUs run N replicas on disjoint inputs with no data collective; the
only cross-rank operations are the barrier and the max-over-ranks timing.  This checks those helpers
with two real processes.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 3.0 if rank == 0 else 5.0  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, dist)
        dist.barrier()
        q.put((rank, tmax, bench.job_value(1e6, tmax, world), bench.rank_info(), bench.rank_seed(1000, rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, value, info, seed in res:
        assert tmax == 5.0                      # both ranks see the slowest rank's time
        assert value == pytest.approx(2 * 1e6 / 5.0)
        assert info[0] == rank and info[1] == 2
    assert res[0][4] != res[1][4]               # replicas denoise different images


def test_single_process_defaults():
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_value(10.0, 2.0, 1) == 5.0
