"""The multi-rank benchmark path on CPU ranks (gloo, world size 2): each rank
renders its own share of the orbit (replicas, no data exchange) and the job
numbers are the slowest rank's time and the summed counts."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    poses = list(range(120))
    share = bench.my_share(poses, rank, world)
    elapsed = 10.0 + 5.0 * rank
    t, (samples, frames) = bench.job_totals(dist, elapsed, [1000 * (rank + 1), len(share)])
    q.put((rank, share, t, samples, frames))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_share_the_orbit_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [r[1] for r in results]
    assert sorted(shares[0] + shares[1]) == list(range(120))
    assert not set(shares[0]) & set(shares[1])
    for _, _, t, samples, frames in results:
        assert t == 15.0                 # the slowest rank's time
        assert samples == 3000           # summed over ranks
        assert frames == 120


def test_single_rank_needs_no_process_group():
    assert bench.my_share(list(range(5)), 0, 1) == list(range(5))
    assert bench.job_totals(None, 3.5, [7, 2]) == (3.5, [7, 2])
