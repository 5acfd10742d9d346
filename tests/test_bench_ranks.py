"""The multi-process side of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job throughput counts every replica, and the
reference arm prints only on rank 0 (no GPU needed)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        out[rank] = ms
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_throughput_counts_every_replica_and_single_process_is_unchanged():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    one = bench.replica_throughput(1, 4 * 2**30, 100.0)
    assert abs(one - 4 * 2**30 / 0.1 / 1e9) < 1e-9
    assert abs(bench.replica_throughput(4, 4 * 2**30, 100.0) - 4 * one) < 1e-9


def test_reference_arm_is_silent_on_other_ranks(capsys):
    import argparse

    ns = argparse.Namespace(n=1 << 22, m=256, k=1024, cond=1e10, passes=3, limbs=[2, 2], steps=1, warmup=0,
                            gpus=2, impl="reference")
    bench.run_reference(ns, rank=1, world=2)
    assert capsys.readouterr().out == ""
