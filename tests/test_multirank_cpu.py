"""Weak-scaling replicas on two CPU ranks (gloo): per-rank inputs and the whole-job aggregate.

The walkers are independent Markov chains, so each rank (one GPU each in production)
evaluates its own batch; the only collective is the max over ranks of the timed region.
These tests run the rank logic of bench.py on CPU with torch.distributed over gloo.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_0908_0681_gb300 import workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seq_seed, move_seeds = bench.rank_seeds(rank, 3)
        w = workloads.five_orbital()
        seqs = workloads.generate_sequences(w, 8, seed=seq_seed)
        digest = float(seqs.tau.sum())
        # pretend timings differ per rank: the aggregate must use the slowest rank
        my_ms = [100.0 * (rank + 1), 7.0 + rank, 3.0]

        def reduce_max(vals):
            t = torch.tensor(vals, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return t.tolist()

        value, t = bench.aggregate(my_ms, 4096, 10, world, reduce_max)
        gathered = [None] * world
        dist.all_gather_object(gathered, (seq_seed, move_seeds, digest))
        q.put((rank, value, t, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_aggregate_on_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # both ranks report the same aggregate, computed from the slowest rank
    (_, v0, t0, g0), (_, v1, t1, g1) = out
    assert v0 == v1 == pytest.approx(2 * 4096 * 10 / 0.2)
    assert t0 == t1 == [200.0, 8.0, 3.0]
    # replicas draw distinct inputs
    assert g0[0][0] != g0[1][0] and g0[0][2] != g0[1][2]
    assert set(g0[0][1]).isdisjoint(g0[1][1])


def test_single_rank_aggregate_needs_no_collective():
    value, t = bench.aggregate([50.0, 1.0, 1.0], 4096, 5, 1, None)
    assert value == pytest.approx(4096 * 5 / 0.05) and t == [50.0, 1.0, 1.0]
