"""The multi-rank logic of bench.py on CPU (gloo, two ranks): the timed
milliseconds are the maximum over the ranks on every rank, the whole-job value
is world x points x steps over that time, and the reference arm runs on rank 0
only (the other ranks exit 0 without work)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 100.0 + 37.5 * rank
    t = bench.reduce_max_ms(mine, world, torch.device("cpu"))
    v = bench.job_throughput(world, 1000, 20, t)
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_max_over_ranks_and_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 100.0 + 37.5 * (world - 1)
    for _, t, v in out:
        assert t == slowest
        assert v == pytest.approx(world * 1000 * 20 / (slowest / 1e3))


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.reduce_max_ms(12.5, 1, None) == 12.5
    assert bench.job_throughput(1, 10, 4, 2.0) == pytest.approx(20000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(impl="reference", workload="mixed", steps=1, warmup=0, precision=None,
                            s_transform="auto", gpus=2, e2e_steps=1, no_cpu_baseline=True, no_context=True)
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""
