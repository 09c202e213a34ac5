"""Multi-rank host logic on CPU: world size 2 over gloo, no GPU.

Each rank takes its block of a seeded instance list, solves it (here with the
CPU oracle, standing in for the per-rank GPU contraction), and the gathered
results must equal a single-process solve of the whole list; the timing
reduction must return the slowest rank's value.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import instances as I
from paper_2008_06888_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_total, q):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = I.mixed_square_batch(n_total, Lmin=2, Lmax=4, seed=9)
    b, e = shard.shard_range(n_total, rank, world)
    local = {}
    for k in range(b, e):
        r = O.solve(insts[k], config=False)
        local[k] = (r["E"], r["count"])
    full = shard.gather_results(local, n_total, rank, world)
    slowest = shard.max_over_ranks(10.0 + rank, world)
    if rank == 0:
        q.put((full, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 5, 16, 17):
        for w in (1, 2, 3, 8):
            parts = [shard.shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and b - a >= d - c
    with pytest.raises(ValueError):
        shard.shard_range(4, 2, 2)


def test_two_ranks_gather_equals_single_process():
    import oracle as O
    n_total = 7
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_total, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    insts = I.mixed_square_batch(n_total, Lmin=2, Lmax=4, seed=9)
    ref = [(O.solve(x, config=False)["E"], O.solve(x, config=False)["count"]) for x in insts]
    assert full == ref
    assert slowest == 11.0
