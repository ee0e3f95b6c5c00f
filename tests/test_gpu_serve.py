"""GPU tests of the serving loop (vr_server_*): frames submitted together are
rendered in batches (one march launch over the tiles of several frames), and each
result must be the same alone and in the mix: bit for bit the image vr_render
gives for that camera and transfer function, which itself matches the oracle."""
import numpy as np
import pytest

import synth
from parity_util import assert_parity
from test_gpu_render import oracle_render

pytestmark = pytest.mark.gpu

RESOLUTIONS = [(64, 48), (96, 96), (160, 90), (200, 150), (37, 61)]


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


def _renderer(vr, torch, cube, tf, cam, brick, precision=0):
    r = vr.VolumeRenderer(0)
    r.load_cube(torch.from_numpy(np.ascontiguousarray(cube)).cuda())
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_camera(cam)
    r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TEX)
    r.set_option(vr.VR_OPT_PRECISION, precision)
    return r


def _requests(shape, n, seed=4):
    """n (camera, transfer function or None) pairs: mixed resolutions and poses,
    every fourth request switching between two transfer functions."""
    rng = np.random.default_rng(seed)
    tfs = [synth.tf_tiny(), synth.make_tf([0.0, 0.0, 0.01, 0.04, 0.1, 0.2, 0.3, 0.5], lo=-3.0, hi=10.0)]
    out = []
    for k in range(n):
        W, H = RESOLUTIONS[k % len(RESOLUTIONS)]
        cam = synth.pose(shape, rng.uniform(0, 2 * np.pi), rng.uniform(-1.0, 1.0), W, H)
        tf = tfs[(k // 4) % 2] if k % 4 == 0 else None
        out.append((cam, tf))
    return out, tfs


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_each_result_is_the_same_alone_and_in_the_mix(vr, torch, precision):
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube = synth.tiny_cube()
    reqs, tfs = _requests(shape, 24)
    # alone: one vr_render per request, the transfer function in force at that point
    alone = []
    with _renderer(vr, torch, cube, tfs[0], reqs[0][0], brick, precision) as r:
        for cam, tf in reqs:
            if tf is not None:
                r.set_transfer_function(tf)
            r.set_camera(cam)
            alone.append(r.render().cpu().numpy())
    # in the mix: all submitted at once
    r = _renderer(vr, torch, cube, tfs[0], reqs[0][0], brick, precision)
    outs = [torch.empty((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda") for cam, _ in reqs]
    with vr.Server(r, 256 << 20, max_batch=8) as srv:
        tickets = [srv.submit(cam, out, tf) for (cam, tf), out in zip(reqs, outs)]
        lat = [srv.wait(t, 60.0) for t in tickets]
        st = srv.stats()
    r.close()
    for k, (a, b) in enumerate(zip(alone, outs)):
        assert np.array_equal(a, b.cpu().numpy()), k
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] < len(reqs)            # frames were batched
    assert all(x >= 0 for x in lat)
    assert max(a[..., 3].max() for a in alone) > 0.3


def test_served_frames_match_the_oracle(vr, torch):
    shape, brick = (64, 64, 64), (32, 32, 32)
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cams = synth.tiny_views()
    r = _renderer(vr, torch, cube, tf, cams[0], brick)
    outs = [torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device="cuda") for c in cams]
    with vr.Server(r, 256 << 20) as srv:
        tickets = [srv.submit(c, o) for c, o in zip(cams, outs)]
        for t in tickets:
            srv.wait(t, 60.0)
    r.close()
    for cam, out in zip(cams, outs):
        ref, amb, _ = oracle_render(cube, tf, cam, brick)
        assert_parity(out.cpu().numpy().astype(np.float64), ref, amb)


def test_admission_by_memory(vr, torch):
    """A frame whose work does not fit half the arena fails on its own (VR_ENOMEM);
    the frames around it are still rendered."""
    shape, brick = (64, 64, 64), (32, 32, 32)
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    small = synth.pose(shape, 0.5, 0.3, 64, 64)
    big = synth.pose(shape, 0.5, 0.3, 2048, 2048)   # ~100k items x 1 KB of fragments > 32 MiB
    r = _renderer(vr, torch, cube, tf, small, brick)
    o1 = torch.empty((64, 64, 4), dtype=torch.float32, device="cuda")
    o2 = torch.empty((2048, 2048, 4), dtype=torch.float32, device="cuda")
    o3 = torch.empty((64, 64, 4), dtype=torch.float32, device="cuda")
    with vr.Server(r, 64 << 20) as srv:
        t1, t2, t3 = srv.submit(small, o1), srv.submit(big, o2), srv.submit(small, o3)
        srv.wait(t1, 60.0)
        with pytest.raises(vr.VRError, match="VR_ENOMEM"):
            srv.wait(t2, 60.0)
        srv.wait(t3, 60.0)
        st = srv.stats()
    r.close()
    assert st["failed"] == 1 and st["completed"] == 2
    assert np.array_equal(o1.cpu().numpy(), o3.cpu().numpy())


def test_transfer_functions_and_thresholds_mix_in_a_batch(vr, torch):
    """Every request switching transfer function (uniform and non-uniform control
    points) and termination threshold: the frames still share batches, and each
    image is vr_render's for its own transfer function and threshold, bit for
    bit."""
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube = synth.tiny_cube()
    tfs = [synth.tf_tiny(),
           synth.make_tf([0.0, 0.0, 0.01, 0.04, 0.1, 0.2, 0.3, 0.5], lo=-3.0, hi=10.0),
           np.array([[-3.0, 0.0, 0.0, 1.0, 0.0], [0.8, 0.1, 0.2, 0.9, 0.0], [1.1, 0.2, 0.6, 0.8, 0.03],
                     [2.9, 0.9, 0.9, 0.9, 0.1], [4.0, 1.0, 0.5, 0.1, 0.3], [9.5, 1.0, 0.0, 0.0, 0.8]])]
    rng = np.random.default_rng(9)
    reqs = []
    for k in range(18):
        cam = synth.pose(shape, rng.uniform(0, 2 * np.pi), rng.uniform(-1.0, 1.0), *RESOLUTIONS[k % 5],
                         term_alpha=(0.99, 0.9, 0.6)[k % 3])
        reqs.append((cam, tfs[(k // 2) % 3]))
    alone = []
    with _renderer(vr, torch, cube, tfs[0], reqs[0][0], brick) as r:
        for cam, tf in reqs:
            r.set_transfer_function(tf)
            r.set_camera(cam)
            alone.append(r.render().cpu().numpy())
    r = _renderer(vr, torch, cube, tfs[0], reqs[0][0], brick)
    outs = [torch.empty((c["height"], c["width"], 4), dtype=torch.float32, device="cuda") for c, _ in reqs]
    with vr.Server(r, 256 << 20, max_batch=8) as srv:
        tickets = [srv.submit(cam, out, tf) for (cam, tf), out in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t, 60.0)
        st = srv.stats()
    r.close()
    for k, (a, o) in enumerate(zip(alone, outs)):
        assert np.array_equal(a, o.cpu().numpy()), k
    assert st["completed"] == len(reqs)
    # thresholds differ between any two consecutive requests (and transfer
    # functions every second one): batches of more than one frame mix them
    assert st["batches"] < len(reqs)
    assert len({float(a[..., 3].max()) for a in alone}) > 3


def test_a_batch_with_many_transfer_functions(vr, torch):
    """Twelve requests with twelve different 40-point transfer functions: the
    batch tables hold up to 512 control points (12 x 41 here, a large shared-memory
    table), and each image is still vr_render's."""
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube = synth.tiny_cube()
    rng = np.random.default_rng(12)
    reqs = []
    for k in range(12):
        alpha = np.sort(rng.uniform(0.0, 0.3, 40))
        alpha[:10] = 0.0
        tf = synth.make_tf(alpha, lo=-3.0 + 0.1 * k, hi=10.0)
        cam = synth.pose(shape, rng.uniform(0, 2 * np.pi), rng.uniform(-1.0, 1.0), 72, 56)
        reqs.append((cam, tf))
    alone = []
    with _renderer(vr, torch, cube, reqs[0][1], reqs[0][0], brick) as r:
        for cam, tf in reqs:
            r.set_transfer_function(tf)
            r.set_camera(cam)
            alone.append(r.render().cpu().numpy())
    r = _renderer(vr, torch, cube, reqs[0][1], reqs[0][0], brick)
    outs = [torch.empty((56, 72, 4), dtype=torch.float32, device="cuda") for _ in reqs]
    with vr.Server(r, 256 << 20, max_batch=16) as srv:
        tickets = [srv.submit(cam, out, tf) for (cam, tf), out in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t, 60.0)
        st = srv.stats()
    r.close()
    assert st["completed"] == 12 and st["failed"] == 0
    for k, (a, o) in enumerate(zip(alone, outs)):
        assert np.array_equal(a, o.cpu().numpy()), k
    assert max(a[..., 3].max() for a in alone) > 0.1


def test_requests_of_different_steps_are_not_batched_together(vr, torch):
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cams = [synth.pose(shape, 0.2 * k, 0.1, 48, 40, step=(0.5 if k % 2 else 0.3)) for k in range(6)]
    alone = []
    with _renderer(vr, torch, cube, tf, cams[0], brick) as r:
        for cam in cams:
            r.set_camera(cam)
            alone.append(r.render().cpu().numpy())
    r = _renderer(vr, torch, cube, tf, cams[0], brick)
    outs = [torch.empty((40, 48, 4), dtype=torch.float32, device="cuda") for _ in cams]
    with vr.Server(r, 128 << 20) as srv:
        ts = [srv.submit(c, o) for c, o in zip(cams, outs)]
        for t in ts:
            srv.wait(t, 60.0)
        st = srv.stats()
    r.close()
    for a, o in zip(alone, outs):
        assert np.array_equal(a, o.cpu().numpy())
    assert st["batches"] == 6   # alternating steps: every frame opens a batch


def test_server_errors_and_shutdown(vr, torch):
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.pose(shape, 0.3, 0.2, 64, 64)
    r = _renderer(vr, torch, cube, tf, cam, brick)
    with pytest.raises(vr.VRError, match="VR_EINVAL"):
        vr.Server(r, 1 << 20)                       # arena too small
    r.set_option(vr.VR_OPT_MODE, 1)
    with pytest.raises(vr.VRError, match="VR_EINVAL"):
        vr.Server(r, 128 << 20)                     # MIP is not served
    r.set_option(vr.VR_OPT_MODE, 0)
    srv = vr.Server(r, 128 << 20)
    with pytest.raises(vr.VRError, match="VR_EINVAL"):
        srv.submit(cam, np.zeros((64, 64, 4), np.float32))   # host output
    outs = [torch.empty((64, 64, 4), dtype=torch.float32, device="cuda") for _ in range(20)]
    for o in outs:
        srv.submit(cam, o)
    srv.close()                                     # finishes the queue, then stops
    ref = outs[0].cpu().numpy()
    assert ref[..., 3].max() > 0.1
    assert all(np.array_equal(ref, o.cpu().numpy()) for o in outs)
    r.close()
