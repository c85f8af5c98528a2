"""The N > 1 path of bench.py (replicas only: N independent copies of the
workload, the slowest rank's step time reported) on world_size-2 gloo
process groups on the CPU; and the reference arm's non-zero ranks exit
without work."""
import argparse
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        out[rank] = bench.slowest_rank_ms(times[rank], world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(3.5, 2.25), (1.0, 7.0)])
def test_slowest_rank_is_reported_on_every_rank(times):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(2, _free_port(), times, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == max(times)


def test_single_rank_reports_its_own_time():
    assert bench.slowest_rank_ms(4.5, 1, "cpu") == 4.5


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="ne_large", steps=2, warmup=3, gpus=2)
    assert bench.run_reference(args) is None  # rank 1 neither builds the graph nor runs the oracle
    assert capsys.readouterr().out == ""
