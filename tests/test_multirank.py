"""Host logic of the multi-rank bench path (independent replicas, weak scaling) on CPU with the gloo backend,
world size 2: the job's time is the maximum over ranks on every rank, the whole-job throughput counts every rank's
DoFs, and non-zero ranks of the reference arm exit without work."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.job_time_ms(torch, dist, 10.0 + 5.0 * rank, torch.device("cpu"), world)
    value = bench.aggregate_gdofs(world, 6_000_000, ms)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_job_time_is_the_max_over_ranks_and_throughput_counts_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, value in res:
        assert ms == 15.0
        assert value == pytest.approx(2 * 6_000_000 / 15e-3 / 1e9)


def test_single_rank_time_is_its_own():
    import bench
    assert bench.job_time_ms(torch, None, 12.5, torch.device("cpu"), 1) == 12.5
    assert bench.aggregate_gdofs(1, 3_000_000, 1.0) == pytest.approx(3.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, impl="reference")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
