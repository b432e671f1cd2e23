"""Multi-process host logic of the benchmark on the CPU (gloo, world size 2): every rank runs its
own design (weak scaling, no data-path collective); the step time is the maximum over ranks and
the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, lr = bench.dist_setup()
    v = bench.reduce_max(10.0 * (rank + 1), torch.device("cpu"))
    q.put((r, ws, lr, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 20.0), (1, 2, 1, 20.0)]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(workload="planar64", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) == 0     # returns without running the oracle


def test_reduce_max_without_a_process_group():
    import torch

    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
