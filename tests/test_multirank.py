"""The multi-rank path of the benchmark on CPU: two gloo ranks, each timing
its own box (weak scaling, no data-path collective), reduce their times to
the slowest rank's and report the whole-job rate; the reference arm does its
work on rank 0 only."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (t, bench.whole_job_rate(128 ** 3, world, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, rate = out[r]
        assert t == 250.0
        assert rate == 2 * 128 ** 3 * 10 / 0.25


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1000, 1, 4, 2.0) == 2e6


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup, n = 2, 1, 3, 8

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
