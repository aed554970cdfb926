"""The benchmark's multi-process path on CPU: two gloo ranks, each an
independent replica, reduce to the whole job's tests (sum) and the slowest
rank's time (max), as bench.py reports them under torchrun."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    tests, ms = bench.reduce_over_ranks(1000.0 * (rank + 1), 10.0 + 5.0 * rank, ws)
    out[rank] = (ws, r, tests, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_sum_of_tests_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        ws, rank, tests, ms = out[r]
        assert (ws, rank) == (world, r)
        assert tests == 3000.0 and ms == 15.0


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.0, 3.0, 1) == (7.0, 3.0)
