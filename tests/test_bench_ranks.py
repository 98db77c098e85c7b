"""The bench's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

The solve does not shard (independent replicas, one per GPU), so the only
cross-rank steps are the barrier around the timed region and the max over
ranks of the elapsed time; the whole-job rate counts every rank's solves.
"""
import argparse
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        # rank r "took" 10 + r seconds
        q.put((rank, bench.max_over_ranks(10.0 + rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 11.0, 1: 11.0}


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks(3.5) == 3.5


def test_replica_rate_counts_every_rank():
    # 2 replicas x 200 solves in 0.5 s (the slowest rank) = 800 solves/s
    assert bench.replica_rate(2, 200, 0.5) == pytest.approx(800.0)
    assert bench.replica_rate(1, 5, 0.0) == 0.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=5, warmup=3, cpu_budget=20.0, gpus=2, impl="reference")
    assert bench.run_reference(args) == 0
