"""Multi-rank path of the benchmark on CPU: two gloo ranks, each with its own
seeded batch of the same shape (weak scaling, no data-path collective); the
only collectives are the timing reductions (max of times, sum of work)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        m = bench.make_workload("pendulum240_x4096", rank, models=4)
        units = float(m.nnz) * 200
        el, km, tot = bench.reduce_across_ranks(100.0 + 10 * rank, 50.0 + rank, units, world, "cpu")
        out[rank] = (el, km, tot, m.nnz, float(m.lower[:1000].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reductions():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
    r0, r1 = out[0], out[1]
    # max over ranks for times, sum over ranks for the work
    assert r0[0] == r1[0] == 110.0 and r0[1] == r1[1] == 51.0
    assert r0[2] == r1[2] == pytest.approx(r0[3] * 200 + r1[3] * 200)
    # same shape on every rank, different seeded data
    assert r0[3] == r1[3]
    assert r0[4] != r1[4]


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_across_ranks(3.0, 2.0, 7.0, 1, "cpu") == (3.0, 2.0, 7.0)
