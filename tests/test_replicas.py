"""The multi-GPU path of the bench is replicas only (independent solves per rank, no data-path
collective): its whole-job figures are the max of the ranks' timed milliseconds and the sum of
their solves.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.replica_totals(10.0 + 3 * rank, 8 * (rank + 1))
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == (13.0, 24.0) and out[1] == (13.0, 24.0)


def test_replica_totals_single_process():
    import bench
    assert bench.replica_totals(7.5, 16) == (7.5, 16.0)


def test_reference_arm_ranks_other_than_zero_do_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(n=1024, warmup=1, steps=1, gpus=2)
    assert bench.run_reference(ns) is None   # returns at once: no oracle work on rank 1
