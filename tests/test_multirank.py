"""The N > 1 launch path of bench.py on CPU: two gloo ranks on 127.0.0.1, each running its own replica
(weak scaling, no data-path collective); the step time is the maximum over ranks and the value counts
the units of all ranks."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    import workloads
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    # each replica draws its own atoms (own seed stream), like run_ours does for rank > 0
    w = workloads.WORKLOADS["c96"]
    rng = np.random.default_rng([w.seed, r])
    pos, _ = workloads.atoms(w, rng if r else None)
    bench.barrier(ws)
    ms = 10.0 + 5.0 * r                       # pretend rank 1 is slower
    t = bench.max_over_ranks(ws, ms)
    out[rank] = (t, float(pos[0, 0]))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_independent_replicas():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0          # max over ranks
    assert out[0][1] != out[1][1]                  # replicas are independent draws


def test_reference_arm_runs_on_rank0_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A(), 2, 1) is None
