"""Host logic of bench.py's multi-process (replica) mode on CPU ranks (gloo):
the max-over-ranks timing, the barrier, and the reference arm's rank-0-only
rule.  The GPU path itself is one independent replica per rank."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        got = bench.aggregate_max(float(10 * (rank + 1)), world, torch.device("cpu"))
        info = bench.dist_info()
        bench.barrier(world)
        q.put((rank, got, info))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_barrier(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, got, info in res:
        assert got == 10.0 * world          # every rank sees the slowest rank's time
        assert info == (rank, world, rank)  # (RANK, WORLD_SIZE, LOCAL_RANK)


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_max(3.5, 1) == 3.5
    bench.barrier(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    class A:  # the fields run_reference reads
        workload, sample, steps, warmup, gpus = "C1", 64, 1, 1, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
