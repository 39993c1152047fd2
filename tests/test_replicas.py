"""The benchmark's multi-process path (one replica per rank, no data-path
collective): on CPU with the gloo backend and two processes, every rank gets
the slowest rank's time and the whole-job value counts the node updates of
all ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    v = bench.job_mlups(1000, 10, world, ms / 1e3)
    q.put((rank, ms, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_share_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, v in res:
        assert ms == 15.0
        assert v == pytest.approx(1000 * 10 * 2 / 0.015 / 1e6)


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_mlups(524288, 2000, 1, 0.15) == pytest.approx(524288 * 2000 / 0.15 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle on the host cores) runs on
    rank 0 alone; the other ranks return at once and print nothing."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=1, warmup=3, cpu_sample_steps=None, drying=False)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
