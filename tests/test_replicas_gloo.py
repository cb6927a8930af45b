"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).  Each rank
runs its own replica (own seeds, no data-path collective); the reported time
is the slowest rank's and the throughput counts every rank's steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        total_ms, value = bench.replica_throughput(my_ms, 10, world, torch.device("cpu"))
        seeds = bench.replica_seeds(rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (total_ms, value, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_seeds():
    port = _free_port()
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total_ms, value, seeds = res[r]
        assert total_ms == 150.0
        assert abs(value - world * 10 / 0.150) < 1e-9
        assert seeds[0] != seeds[1] and seeds[0][0] != seeds[1][0]


def test_reference_arm_other_ranks_exit_without_work(capsys):
    import argparse
    import bench
    args = argparse.Namespace(workload="c1_10k_128", steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
