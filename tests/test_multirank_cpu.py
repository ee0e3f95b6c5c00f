"""Multi-rank paths on CPU ranks (gloo).

* The benchmark's replicas (world size 2): each rank renders its own share of
  the orbit (no data exchange); the job numbers are the slowest rank's time and
  the summed counts.
* Sort-last distribution of one frame (Sections 2.3.1, 2.3.3, 2.3.4; world
  sizes 2 and 3): each rank sends its k-d leaf's rectangle-clipped sub-image to
  the root, which folds them in visibility order; and a rank that leaves before
  the exchange makes the root raise instead of hanging.
"""
import os
import socket
import time

import numpy as np
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


# ---------------------------------------------------------------- sort-last exchange

SHARD_SHAPE, SHARD_BRICK = (64, 64, 64), (16, 16, 16)


def _shard_case():
    import synth
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=72, height=60)[1]
    return cube, tf, cam


def _leaf_map(world):
    """Region (leaf number) of every brick for a world-size partition."""
    from paper_1205_0282_gb300 import shard
    R = shard.leaf_ranges(SHARD_SHAPE, SHARD_BRICK, world)
    nb = [(n - 1 + b - 1) // b for n, b in zip(SHARD_SHAPE, SHARD_BRICK)]
    ids = np.arange(nb[0] * nb[1] * nb[2])
    idx = np.stack([ids % nb[0], (ids // nb[0]) % nb[1], ids // (nb[0] * nb[1])], axis=1)
    reg = -np.ones(len(ids), dtype=np.int32)
    for k, r in enumerate(R):
        inside = ((idx >= r[:3]) & (idx < r[3:])).all(axis=1)
        reg[inside] = k
    return R, reg


def _rank_subimage(rank, world):
    """This rank's rect and sub-image, computed by the oracle (the CPU stand-in for
    vr_render_rect on the rank's leaf)."""
    import oracle
    import torch
    from paper_1205_0282_gb300 import vr
    cube, tf, cam = _shard_case()
    R, reg = _leaf_map(world)
    rect = vr.vr_plan_region_rect(cam, SHARD_SHAPE, SHARD_BRICK, R[rank, :3], R[rank, 3:])
    x0, y0, x1, y1 = (int(v) for v in rect)
    if x1 < x0 or y1 < y0:
        return rect, None
    jj, ii = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
    own = np.where(reg == rank, 0, -1).astype(np.int32)
    rgba, _, _ = oracle.render(cube, tf, cam, brick=SHARD_BRICK, pixels=(jj * cam["width"] + ii).reshape(-1),
                               regions=own)
    return rect, torch.from_numpy(rgba.astype(np.float32).reshape(y1 - y0 + 1, x1 - x0 + 1, 4))


def _exit(q, code):
    """Leave the process at once, after the queue has delivered its messages."""
    q.close()
    q.join_thread()
    os._exit(code)


def _shard_rank(rank, world, port, q, fail_rank, fail_mode):
    import datetime

    import torch.distributed as dist
    from paper_1205_0282_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == fail_rank:
        # a rank that fails before the exchange: it leaves, or stalls, without sending
        q.put((rank, fail_mode, None))
        if fail_mode == "stalls":
            time.sleep(8)
        _exit(q, 3)
    rect, sub = _rank_subimage(rank, world)
    t0 = time.monotonic()
    try:
        got = shard.exchange_subimages(dist, rank, world, rect, sub, timeout_s=5.0)
    except Exception as e:  # noqa: BLE001 - reported to the test
        q.put((rank, "error", (type(e).__name__, time.monotonic() - t0)))
        _exit(q, 0)
    if rank == 0:
        q.put((rank, "ok", [(g[0].tolist(), None if g[1] is None else g[1].numpy()) for g in got]))
    else:
        q.put((rank, "ok", None))
    dist.barrier()
    dist.destroy_process_group()


def _run_shard(world, fail_rank=-1, fail_mode=""):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q, fail_rank, fail_mode))
             for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(world):
        rank, status, payload = q.get(timeout=180)
        results[rank] = (status, payload)
    for p in procs:
        p.join(timeout=60)
    return results, [p.exitcode for p in procs]


def _fold(images, rects, W, H, tau):
    acc = np.zeros((H, W, 4))
    for im, (x0, y0, x1, y1) in zip(images, rects):
        if im is None:
            continue
        a = acc[y0:y1 + 1, x0:x1 + 1]
        live = a[..., 3:4] < tau
        a += np.where(live, (1.0 - a[..., 3:4]) * im, 0.0)
    return acc


@pytest.mark.parametrize("world", [2, 3])
def test_sort_last_exchange_and_root_fold(world):
    """CPU ranks (gloo): each rank sends its leaf's rect-clipped sub-image to the
    root, which folds them in the leaves' visibility order; the result is the
    oracle's two-level render of the same partition."""
    import oracle
    from paper_1205_0282_gb300 import shard
    results, codes = _run_shard(world)
    assert codes == [0] * world
    status, got = results[0]
    assert status == "ok"
    cube, tf, cam = _shard_case()
    order = shard.visibility_order(SHARD_SHAPE, SHARD_BRICK, world, cam["eye"])
    images = [got[k][1] for k in order]
    rects = [got[k][0] for k in order]
    assert sum(im is not None for im in images) >= 2
    frame = _fold(images, rects, cam["width"], cam["height"], cam["term_alpha"])
    _, reg = _leaf_map(world)
    ref, amb, _ = oracle.render(cube, tf, cam, brick=SHARD_BRICK, regions=reg)
    ok = amb == 0
    assert np.abs(frame - ref)[ok].max() < 1e-6
    assert ref[..., 3].max() > 0.3


@pytest.mark.parametrize("mode", ["left", "stalls"])
def test_a_failed_rank_makes_the_root_fail_not_hang(mode):
    """The failure is made on the host: rank 1 exits, or stays alive without
    sending; the root's receive raises (connection closed, or the 5 s exchange
    timeout) and the root returns."""
    results, codes = _run_shard(2, fail_rank=1, fail_mode=mode)
    assert results[1][0] == mode and codes[1] == 3
    status, payload = results[0]
    assert status == "error", results[0]
    assert payload[1] < (2.0 if mode == "left" else 15.0)
    if mode == "stalls":
        assert payload[1] >= 4.5
