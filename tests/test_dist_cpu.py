"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2):
replicas only -- the slowest rank's time and the sum of all ranks' site
updates make the whole-job figure; the reference arm prints on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    times, counts = bench.reduce_over_ranks([10.0 + rank, 5.0 * (rank + 1)], [100.0 * (rank + 1), 7.0], "cpu", world)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (times, counts)


def test_reduce_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        times, counts = res[rank]
        assert times == [11.0, 10.0]          # max over ranks
        assert counts == [300.0, 14.0]        # sum over ranks


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_over_ranks([3.0], [4.0], "cpu", 1) == ([3.0], [4.0])


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.reference_arm(argparse.Namespace(gpus=2, steps=1, warmup=0))
    assert capsys.readouterr().out == ""
