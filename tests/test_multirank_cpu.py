"""The N > 1 bench plumbing on CPU (gloo, world_size 2): each rank draws its own batch
(replicas over independent problems, weak scaling), the job time is the slowest rank's and
the pair count the sum; the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ops = bench._workload_ops(rank)
        first = float(ops[0].P[0, 0])
        ms, pairs = bench.reduce_time_pairs(100.0 + 50.0 * rank, 1000 + rank, world, "cpu")
        firsts = [None] * world
        dist.all_gather_object(firsts, first)
        out[rank] = (ms, pairs, firsts)
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_and_independent_batches():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, pairs, firsts = res[rank]
        assert ms == 150.0            # the slowest rank
        assert pairs == 2001.0        # all ranks' pairs
        assert firsts[0] != firsts[1]  # each rank draws its own problems


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, cpu_sample_ops=1))
    assert capsys.readouterr().out == ""
