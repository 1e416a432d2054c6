"""Host logic of bench.py's multi-rank (replica) path on CPU: two gloo ranks reduce their
timings to the slowest rank's, the job's throughput is the sum over replicas at that time,
and the reference arm runs on rank 0 only.  No GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]                      # per-rank device time of a step
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.aggregate_rate(world, 1 << 20, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{slowest} {rate}")


def test_two_gloo_ranks_reduce_to_the_slowest(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        slowest, rate = map(float, open(tmp_path / f"rank{rank}.txt").read().split())
        assert slowest == 20.0
        assert rate == pytest.approx(2 * (1 << 20) / 20e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
