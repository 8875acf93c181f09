"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank runs its own
independent replica, and the reported time is the max over ranks. No GPU, no collective
on the data path."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r pretends its timed region took (10 + r) ms and its e2e region (20 - r) ms
        total, e2e = bench.combine_over_ranks([10.0 + rank, 20.0 - rank], world)
        out[rank] = (total, e2e, bench.replica_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_independent_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][:2] == (11.0, 20.0) and res[1][:2] == (11.0, 20.0)
    assert res[0][2] != res[1][2]  # distinct swarms per rank


def test_whole_job_throughput_counts_every_rank():
    # 65536 drones x 5 substeps per rank, 2 ranks, 10 steps in 1 ms (max over ranks)
    assert bench.throughput(65536 * 5, 2, 10, 1.0) == pytest.approx(65536 * 5 * 2 * 10 / 1e-3)
    assert bench.combine_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
