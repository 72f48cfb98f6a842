"""The bench's multi-rank bookkeeping, run as two gloo ranks on the CPU:
time is the slowest rank's, lattice updates add up over ranks (N GPUs run
independent replicas, weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, lups = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
        out[rank] = (ms, lups)
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (150.0, 3000.0)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_over_ranks(12.5, 7, torch.device("cpu")) == (12.5, 7.0)
