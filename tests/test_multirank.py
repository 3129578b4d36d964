"""The multi-rank bench path on CPU: two gloo ranks, each timing its own
frame; the job rate uses the slowest rank (no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, results):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    dist.barrier()
    own = [0.5, 0.8][rank]  # rank 1 is slower
    slowest = bench.max_over_ranks(own, ws)
    results[rank] = (slowest, bench.aggregate_rate(8_589_934_592, 10, ws, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    manager = mp.Manager()
    results = manager.dict()
    mp.spawn(_rank, args=(ws, _free_port(), results), nprocs=ws, join=True)
    for r in range(ws):
        slowest, rate = results[r]
        assert slowest == pytest.approx(0.8)
        assert rate == pytest.approx(2 * 8_589_934_592 * 10 / 0.8 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.aggregate_rate(100, 2, 1, 1.0) == pytest.approx(2e-7)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the FP64 oracle on the host cores)
    runs on rank 0 alone; other ranks exit 0 without work or output."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(gpus=2, steps=3, warmup=3, impl="reference")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
