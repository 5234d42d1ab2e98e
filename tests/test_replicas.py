"""Multi-rank path of the bench on the CPU: independent replicas, one process
per rank, joined only by the timing reduction (gloo, world size 2)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2111_13072_gb300.inputs import WORKLOADS, workload_state
from paper_2111_13072_gb300.replicas import max_over_ranks, rank_seed, throughput


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = WORKLOADS["fp64_n2e4_l8"]
        seed = rank_seed(w.seed, rank)
        x, _ = workload_state(w.__class__(**{**w.__dict__, "seed": seed}), N=64)
        local = [1.0 + rank, 10.0 - rank]          # this rank's (step, e2e) times
        red = max_over_ranks(local, dist)
        # each rank reports its first particle, to show the instances differ
        mine = torch.tensor(x[0], dtype=torch.float64)
        allx = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allx, mine)
        out[rank] = (seed, red, [a.tolist() for a in allx])
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_the_slowest_time_and_run_distinct_replicas():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    seeds = [out[r][0] for r in range(world)]
    assert seeds == [0, 1]
    for r in range(world):
        assert out[r][1] == [2.0, 10.0]          # maximum over ranks, element-wise
    firsts = out[0][2]
    assert not np.allclose(firsts[0], firsts[1])  # the replicas are independent instances
    # whole-job throughput: all ranks' particle-steps over the slowest rank's time
    assert throughput(2_000_000, 100, world, 0.2) == pytest.approx(2e6 * 100 * 2 / 0.2)


def test_single_process_reduction_is_the_identity():
    assert max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert rank_seed(7, 0) == 7
