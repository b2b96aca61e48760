"""The bench's N > 1 path on the CPU: world_size-2 gloo ranks, no GPU.

With one matrix per GPU there is no exchange step, so `bench.py --gpus N` runs N
independent replicas: every rank times its own steps, the time is the maximum over ranks
(all-reduce MAX), barriers bracket the timed region, and the whole-job value counts the
bytes of all ranks. These tests run that host logic over gloo on two CPU processes, and
check that the reference arm does its work on rank 0 only.
"""
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


def _rank_main(rank: int, world: int, port: int, steps: int):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        assert (w, r, local) == (world, rank, rank)
        bench.barrier(world)
        # each rank's own time; the job is timed by the slowest rank
        mine = 0.5 + 0.25 * rank
        slowest = bench.reduce_max(mine, world, torch.device("cpu"))
        assert slowest == 0.5 + 0.25 * (world - 1)
        bench.barrier(world)
        value = bench.replica_throughput(world, 2.0e9, steps, slowest)
        assert value == pytest.approx(world * 2.0e9 * steps / slowest / 1e9)
        # every rank computes the same whole-job value
        t = torch.tensor([value], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        assert t.item() == value
    finally:
        dist.destroy_process_group()


def test_replicas_over_gloo_take_the_slowest_rank():
    mp.spawn(_rank_main, args=(2, _free_port(), 10), nprocs=2, join=True)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.reduce_max(3.5, 1, None) == 3.5
    bench.barrier(1)
    assert bench.replica_throughput(1, 1e9, 4, 2.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # under torchrun the other ranks of the reference arm exit 0 without work (no workload is built)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "build_workload", lambda name: (_ for _ in ()).throw(AssertionError("built")))

    class Args:
        workload = "q1v_96"
        steps = 1
        warmup = 0

    assert bench.run_reference(Args()) == 0
