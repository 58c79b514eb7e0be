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
    cls = (4, 2, 4, 6)          # diagonal, single-phase, general, control-carrying entries
    per_term = 2 * 4 + 4 * 2 + 8 * 4 + 4 * 4   # per column: the product and the row update (d = 4)
    # forward and costate chain: sum s m terms
    assert bench.forward_flops(m, s, cls, dim=4, n=2) == (3 + 4) * per_term * 2
    assert bench.costate_flops(m, s, cls, dim=4, n=2) == (3 + 4) * per_term * 2
    # gradient: m s control accumulations and m s - 1 products per step
    assert bench.gradient_flops(m, s, cls, dim=4, n=2) == 2 * ((3 * 8 * 6 + 2 * per_term) + (4 * 8 * 6 + 3 * per_term))
    # fused backward: per substep (3m - 1) products + m control accumulations
    want = 2 * (1 * (8 * per_term + 3 * 8 * 6) + 2 * (5 * per_term + 2 * 8 * 6))
    assert bench.fused_backward_flops(m, s, cls, dim=4, n=2) == want


def test_entry_classes_of_a_two_level_drive():
    """H0 = (delta/2) sigma_z (real diagonal), one control sigma_x (real off-diagonal: single phase)."""
    import bench
    from workloads import two_level_rabi
    p = two_level_rabi(3, 0.1, delta=1.0)
    n_diag, n_single, n_general, n_ctrl = bench.entry_classes(p)
    assert (n_diag, n_single, n_general, n_ctrl) == (2, 2, 0, 2)


def test_single_rank_aggregate_without_collectives():
    import bench
    v, t = bench.aggregate(4.0, 8, 1)
    assert (v, t) == (2.0, 4.0)
