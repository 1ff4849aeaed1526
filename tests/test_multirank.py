"""The multi-GPU path of bench.py is replicas only: each rank separates its
own job and the ranks meet only at the barrier and the max-over-ranks
reduction of the timed region.  Exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 150.0][rank]
        slowest = bench.max_over_ranks(elapsed, world)
        bench.barrier(world)
        value = bench.aggregate(3000 * 50, 4, world, slowest)
        q.put((rank, bench.job_seed(rank), slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas(repo_root):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    seeds = [o[1] for o in out]
    assert len(set(seeds)) == 2                       # distinct jobs per rank
    assert all(o[2] == 150.0 for o in out)            # slowest rank's time on every rank
    expected = 2 * 3000 * 50 * 4 / 0.150
    assert all(abs(o[3] - expected) < 1e-6 * expected for o in out)
