"""GPU parity of the sort-last distribution (Sections 2.3.1, 2.3.3, 2.3.4):
rectangle-clipped renders, per-leaf sub-images, the root's fold as virtual ranks
on one GPU (one stream per rank), and the same over gloo ranks in separate
processes, all against the FP64 oracle's two-level fold."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


def _renderer(vr, torch, cube, tf, cam, brick, kernel=None):
    r = vr.VolumeRenderer(0)
    r.load_cube(torch.from_numpy(np.ascontiguousarray(cube)).cuda())
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_camera(cam)
    if kernel is not None:
        r.set_option(vr.VR_OPT_KERNEL, kernel)
    return r


def _leaf_map(shape, brick, R):
    nb = [(n - 1 + b - 1) // b for n, b in zip(shape, brick)]
    ids = np.arange(nb[0] * nb[1] * nb[2])
    idx = np.stack([ids % nb[0], (ids // nb[0]) % nb[1], ids // (nb[0] * nb[1])], axis=1)
    reg = -np.ones(len(ids), dtype=np.int32)
    for k, r in enumerate(R):
        reg[((idx >= r[:3]) & (idx < r[3:])).all(axis=1)] = k
    return reg


@pytest.mark.parametrize("kernel", [2, 1, 0])   # texture, direct, TMA
def test_render_rect_is_the_crop_of_the_full_render(vr, torch, kernel):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=101, height=77)[2]
    with _renderer(vr, torch, cube, tf, cam, (16, 16, 16), kernel) as r:
        full = r.render().cpu().numpy()
        for rect in [(0, 0, 100, 76), (3, 5, 50, 41), (17, 9, 17, 60), (90, 70, 100, 76), (40, 0, 99, 0)]:
            x0, y0, x1, y1 = rect
            sub = r.render_rect(rect).cpu().numpy()
            # a rectangle can drop bricks whose fragments are exactly zero; the
            # composite's shuffle scan groups fragments in fours, so the 'over'
            # products may regroup: equal up to one FP32 ulp of values <= 1
            assert np.abs(sub - full[y0:y1 + 1, x0:x1 + 1]).max() <= 1.2e-7, rect
            host = np.zeros_like(sub)
            vr.vr_render_rect(r.ctx, rect, host)
            assert np.array_equal(host, sub)
        assert r.render_rect((5, 5, 4, 9)) is None   # empty


@pytest.mark.parametrize("parts", [2, 3])
def test_leaf_subimages_match_the_oracle(vr, torch, parts):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    shape, brick = (64, 64, 64), (16, 16, 16)
    cam = synth.tiny_views(width=96, height=80)[0]
    R = vr.vr_kd_partition(shape, brick, parts)
    reg = _leaf_map(shape, brick, R)
    with _renderer(vr, torch, cube, tf, cam, brick) as r:
        for k in range(parts):
            r.set_region(R[k, :3], R[k, 3:])
            rect = r.region_rect()
            assert rect.tolist() == vr.vr_plan_region_rect(cam, shape, brick, R[k, :3], R[k, 3:]).tolist()
            x0, y0, x1, y1 = (int(v) for v in rect)
            sub = r.render_rect(rect).cpu().numpy().astype(np.float64)
            jj, ii = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
            ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, pixels=(jj * cam["width"] + ii).reshape(-1),
                                        regions=np.where(reg == k, 0, -1), amb_alpha=AMB_ALPHA,
                                        amb_steps=AMB_STEPS)
            assert_parity(sub.reshape(-1, 4), ref, amb)


def _virtual_ranks(vr, torch, r, shape, brick, cam, parts):
    """One frame as `parts` virtual ranks on one GPU: rank k renders leaf k on its
    own stream; the root stream waits for all of them and folds in visibility order."""
    R = vr.vr_kd_partition(shape, brick, parts)
    streams = [torch.cuda.Stream() for _ in range(parts)]
    subs, rects = [], []
    for k in range(parts):
        r.set_region(R[k, :3], R[k, 3:])
        rect = r.region_rect()
        with torch.cuda.stream(streams[k]):
            sub = r.render_rect(rect, stream=streams[k])
        subs.append(sub)
        rects.append(rect)
    root = torch.cuda.current_stream()
    for s in streams:
        root.wait_stream(s)
    order = vr.vr_kd_order(shape, brick, parts, cam["eye"])
    frame = r.composite([subs[k] for k in order], np.stack([rects[k] for k in order]))
    torch.cuda.synchronize()
    return frame.cpu().numpy().astype(np.float64), R


@pytest.mark.parametrize("parts", [2, 3, 5, 8])
@pytest.mark.parametrize("view", [0, 3])
def test_virtual_ranks_on_one_gpu(vr, torch, parts, view):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    shape, brick = (64, 64, 64), (16, 16, 16)
    cam = synth.tiny_views(width=128, height=112)[view]
    with _renderer(vr, torch, cube, tf, cam, brick) as r:
        frame, R = _virtual_ranks(vr, torch, r, shape, brick, cam, parts)
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, regions=_leaf_map(shape, brick, R),
                                amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert_parity(frame, ref, amb)


def test_virtual_ranks_without_termination_equal_the_single_render(vr, torch):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    shape, brick = (64, 64, 64), (16, 16, 16)
    cam = synth.tiny_views(width=128, height=112, term_alpha=1.0)[1]
    with _renderer(vr, torch, cube, tf, cam, brick) as r:
        whole = r.render().cpu().numpy().astype(np.float64)
        frame, _ = _virtual_ranks(vr, torch, r, shape, brick, cam, 4)
    assert np.abs(frame - whole).max() < 2e-6
    assert whole[..., 3].max() > 0.3


def test_virtual_ranks_ragged_eye_inside(vr, torch):
    shape, brick = (61, 47, 53), (24, 16, 20)
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.camera((30.0, 20.0, 25.0), (60.0, 40.0, 0.0), (0, 1, 0), 80.0, 90, 70)
    with _renderer(vr, torch, cube, tf, cam, brick) as r:
        frame, R = _virtual_ranks(vr, torch, r, shape, brick, cam, 3)
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, regions=_leaf_map(shape, brick, R),
                                amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert_parity(frame, ref, amb)


def test_composite_outputs_and_errors(vr, torch):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=40, height=30)[0]
    with _renderer(vr, torch, cube, tf, cam, (16, 16, 16)) as r:
        a = r.render_rect((0, 0, 19, 29))
        b = r.render_rect((10, 5, 39, 29))
        dev = r.composite([a, None, b], [(0, 0, 19, 29), (0, 0, -1, -1), (10, 5, 39, 29)]).cpu().numpy()
        host = np.zeros((30, 40, 4), dtype=np.float32)
        vr.vr_composite_subimages(r.ctx, [a, None, b], [(0, 0, 19, 29), (0, 0, -1, -1), (10, 5, 39, 29)], host)
        assert np.array_equal(dev, host)
        an, bn = a.cpu().numpy(), b.cpu().numpy()
        assert np.array_equal(dev[:, 20:], np.pad(bn, ((5, 0), (0, 0), (0, 0)))[:, 10:])
        assert np.array_equal(dev[:5, :20], an[:5])
        empty = r.composite([], np.zeros((0, 4), np.int32)).cpu().numpy()
        assert not empty.any()
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.composite([a], [(0, 0, 40, 29)])
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.render_rect((0, 0, 40, 10))
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.set_region((0, 0, 0), (5, 4, 4))
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.composite([a] * 257, [(0, 0, 19, 29)] * 257)


# ------------------------------------------------------------ gloo ranks, one GPU

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gpu_rank(rank, world, port, q):
    import datetime

    import torch
    import torch.distributed as dist
    from paper_1205_0282_gb300 import shard, vr
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=96, height=80)[2]
    r = _renderer(vr, torch, cube, tf, cam, (16, 16, 16))
    frame = shard.render_distributed(r, dist, rank, world)
    q.put((rank, None if frame is None else frame.cpu().numpy()))
    r.close()
    dist.barrier()
    dist.destroy_process_group()


def test_render_distributed_over_gloo_ranks(vr):
    """Two processes on the one GPU, exchanging host copies of their sub-images
    over gloo (no kernel waits on another process)."""
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[1] is None
    frame = got[0].astype(np.float64)
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=96, height=80)[2]
    shape, brick = (64, 64, 64), (16, 16, 16)
    R = vr.vr_kd_partition(shape, brick, world)
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, regions=_leaf_map(shape, brick, R),
                                amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert_parity(frame, ref, amb)
