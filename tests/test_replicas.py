"""The multi-GPU path of the benchmark is replicas only: one process per GPU,
each solving the workload on its own, joined by a barrier and by the maximum
of their times (the job ends with its slowest replica).  This runs that host
logic (bench.max_over_ranks) as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 3.0 * rank          # rank 1 is the slow replica
        got = bench.max_over_ranks(mine)  # CPU tensors: the gloo backend
        dist.barrier()
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_replica_times_reduce_to_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert dict(out) == {0: 13.0, 1: 13.0}


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench

    if dist.is_initialized():
        pytest.skip("a process group is already running")
    assert bench.max_over_ranks(4.5) == 4.5
