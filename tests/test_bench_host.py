"""Host logic of bench.py: the whole-job aggregation over ranks (gloo, world size 2, CPU) and the work model."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def rmax(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def rsum(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    local_seconds = 2.0 + rank          # rank 1 is the slowest
    value, tmax = bench.aggregate(local_seconds, 5, world, rmax, rsum)
    out[rank] = (value, tmax, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sums_units_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        value, tmax, env = out[r]
        assert tmax == 3.0
        assert value == pytest.approx(10 / 3.0)
        assert env == (2, r, r)


def test_work_model_counts():
    import bench
    m = np.array([3, 2])
    s = np.array([1, 2])
    # forward: sum s m terms, each 8 nnz n + 4 d n flops
    assert bench.forward_flops(m, s, nnz=10, dim=4, n=2) == (3 + 4) * (8 * 10 * 2 + 4 * 4 * 2)
    # backward: per substep (3m - 1) sparse products + m W-accumulations on control entries
    want = 1 * (8 * (160 + 32) + 3 * 8 * 6 * 2) + 2 * (5 * (160 + 32) + 2 * 8 * 6 * 2)
    assert bench.backward_flops(m, s, nnz=10, nnz_ctrl_entries=6, dim=4, n=2) == want


def test_single_rank_aggregate_without_collectives():
    import bench
    v, t = bench.aggregate(4.0, 8, 1)
    assert (v, t) == (2.0, 4.0)
