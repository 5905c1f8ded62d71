"""Replicas-only multi-process path on CPU (gloo, world size 2).

The counting path does not shard: every rank counts its own replica of the
workload, with no collective on the data path.  What the ranks share is the
timing: the slowest rank's time sets the job's time and the job's rate is
world x units / that time.  These tests run that host logic over a real
two-process group.
"""
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
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle
    from paper_1506_04322_gb300 import inputs

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # each replica times its own copy; rank 1 is the slow one
        slow = bench.max_over_ranks(10.0 + 5.0 * rank)
        rate = bench.job_rate(1000, world, slow / 1000.0)
        # replicas of the same seeded workload give the same counts
        g = inputs.erdos_renyi(60, 0.15, 17)
        counts = oracle.o2_global(g)
        gathered = [None] * world
        dist.all_gather_object(gathered, [str(c) for c in counts])
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{slow} {rate} {int(all(x == gathered[0] for x in gathered))}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        slow, rate, same = open(tmp_path / f"rank{r}.txt").read().split()
        assert float(slow) == 15.0                  # max over ranks, seen by every rank
        assert float(rate) == pytest.approx(2 * 1000 / 0.015)
        assert same == "1"


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(10, 1, 2.0) == 5.0
