"""GPU parity of the out-of-core path (vr_load_cube_host): the cube stays in host
memory, bricks are copied into a device cache under a memory budget and marched
from there, by the texture march on layered copies of the cache's slots
(VR_OPT_OOC_MARCH 1, the default) or by the direct march on the blocks (0).
Its images must equal the in-core march of the same kernel bit for bit (same
voxels, same arithmetic) and match the FP64 oracle; the residency counters must
show reuse when the frame fits the cache and streaming when it does not."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity
from ooc_budget import budget_for
from test_gpu_render import RAGGED, oracle_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


def _incore(vr, torch, cube, tf, cam, brick, mode=0, march=1):
    """In-core render with the kernel the out-of-core march mirrors."""
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(np.ascontiguousarray(cube)).cuda())
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TEX if march else vr.VR_KERNEL_DIRECT)
        r.set_option(vr.VR_OPT_MODE, mode)
        return r.render().cpu().numpy()


def _ooc(vr, cube, tf, brick, budget_bricks=0, mode=0, march=1):
    """Out-of-core context whose cache holds budget_bricks slots (the texture march
    keeps three layered copies of each slot, or with march 3 the one along z, plus
    a staging area for one launch's blocks)."""
    r = vr.VolumeRenderer(0)
    r.load_cube_host(cube)
    r.set_option(vr.VR_OPT_OOC_MARCH, march)
    if budget_bricks:
        r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget_for(budget_bricks, brick, march))
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_option(vr.VR_OPT_MODE, mode)
    return r


@pytest.mark.parametrize("march", [1, 0])
@pytest.mark.parametrize("budget", [0, 20, 9, 2])
@pytest.mark.parametrize("view", [0, 2])
def test_out_of_core_equals_in_core(vr, torch, budget, view, march):
    """Same image as the in-core march of the same kernel, frame after frame.  A
    frame whose bricks fit uploads them once; a larger one keeps S - 2H bricks
    resident (S slots, H = clamp(S / 8, 1, 32)) and streams the rest through the
    ring."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)    # 64 bricks
    cam = synth.tiny_views(width=96, height=80)[view]
    ref = _incore(vr, torch, cube, tf, cam, brick, march=march)
    ups = []
    with _ooc(vr, cube, tf, brick, budget, march=march) as r:
        r.set_camera(cam)
        for _ in range(3):
            r.reset_stats()
            img = r.render().cpu().numpy()
            assert np.array_equal(img, ref)
            st = r.stats()
            assert st["device_errors"] == 0
            assert st["bricks_uploaded"] + st["bricks_cached"] == st["bricks_rendered"]
            ups.append(st["bricks_uploaded"])
        P = st["bricks_rendered"]
    S = budget if budget else 64
    assert ups[0] == P
    if P <= S:
        assert ups[1] == ups[2] == 0
    else:
        H = max(1, min(S // 8, 32))
        assert ups[1] == ups[2] == P - (S - 2 * H)


def test_cache_evicts_least_recently_used(vr, torch):
    """A cache that holds either view's bricks but not both: going back to the
    first view re-uploads exactly the bricks the second view evicted."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)
    # the eye inside the cube, looking at opposite corners: each view misses the
    # bricks behind it
    a = synth.camera((33.0, 31.0, 32.5), (63.0, 63.0, 63.0), (0, 1, 0), 40.0, 64, 64)
    b = synth.camera((33.0, 31.0, 32.5), (0.0, 0.0, 0.0), (0, 1, 0), 40.0, 64, 64)
    counts = {}
    with _ooc(vr, cube, tf, brick) as r:     # every brick fits: learn each view's brick count
        for name, cam in (("a", a), ("b", b)):
            r.set_camera(cam)
            r.reset_stats()
            r.render()
            counts[name] = r.stats()["bricks_rendered"]
    budget = max(counts.values())
    assert budget < 64
    with _ooc(vr, cube, tf, brick, budget) as r:
        ups = []
        for cam in (a, b, a):
            r.set_camera(cam)
            r.reset_stats()
            img = r.render().cpu().numpy()
            st = r.stats()
            ups.append(st["bricks_uploaded"])
            assert st["bricks_uploaded"] + st["bricks_cached"] == st["bricks_rendered"]
        assert np.array_equal(img, _incore(vr, torch, cube, tf, a, brick))
    assert ups[0] == counts["a"]
    assert 0 < ups[2] <= ups[1]          # evicted bricks come back, resident ones do not


def test_out_of_core_matches_the_oracle(vr):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    for view in range(4):
        cam = synth.tiny_views()[view]
        with _ooc(vr, cube, tf, (32, 32, 32), 3) as r:
            r.set_camera(cam)
            img = r.render().cpu().numpy().astype(np.float64)
        ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
        assert_parity(img, ref, amb)


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:3])
def test_out_of_core_ragged(vr, shape, brick, camk, step, tau):
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    with _ooc(vr, cube, tf, brick, 5) as r:
        r.set_camera(cam)
        img = r.render().cpu().numpy().astype(np.float64)
        host = np.zeros_like(img, dtype=np.float32)
        r.render(host)
    assert np.array_equal(host.astype(np.float64), img)
    ref, amb, _ = oracle_render(cube, tf, cam, brick)
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("march", [1, 0])
def test_out_of_core_mip(vr, torch, march):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=80, height=72)[1]
    ref = _incore(vr, torch, cube, tf, cam, (16, 16, 16), mode=1, march=march)
    with _ooc(vr, cube, tf, (16, 16, 16), 6, mode=1, march=march) as r:
        r.set_camera(cam)
        assert np.array_equal(r.render().cpu().numpy(), ref)


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_out_of_core_texture_march_dynamic_step(vr, torch, shape, brick, camk, step, tau):
    """The dynamic step on the slot copies: the in-core texture march's image, and
    the oracle's."""
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(np.ascontiguousarray(cube)).cuda())
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TEX)
        r.set_option(vr.VR_OPT_STEP_MODE, 1)
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        ref_gpu = r.render().cpu().numpy()
    with _ooc(vr, cube, tf, brick, 4) as r:
        r.set_option(vr.VR_OPT_STEP_MODE, 1)
        r.set_camera(cam)
        img = r.render().cpu().numpy()
    assert np.array_equal(img, ref_gpu)
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS, step_mode=1)
    assert_parity(img.astype(np.float64), ref, amb)


@pytest.mark.parametrize("march", [3, 4])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("budget", [0, 20, 5])
def test_out_of_core_single_copy_march(vr, budget, mode, march):
    """VR_OPT_OOC_MARCH 3: the texture march on one layered copy of the slots,
    layers along z; 4: on the two copies along x and z.  The same samples as the
    three-copy march, gathered in another plane where a ray's dominant axis has no
    copy: within FP32 rounding of its image (emission-absorption and MIP), frame
    after frame with every brick resident or streamed, and oracle parity."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)
    for view in (0, 2):
        cam = synth.tiny_views(width=96, height=80)[view]
        with _ooc(vr, cube, tf, brick, budget, mode=mode, march=1) as r:
            r.set_camera(cam)
            want = r.render().cpu().numpy().astype(np.float64)
        with _ooc(vr, cube, tf, brick, budget, mode=mode, march=march) as r:
            r.set_camera(cam)
            for k in range(3):
                r.reset_stats()
                img = r.render().cpu().numpy().astype(np.float64)
                assert np.abs(img - want).max() <= 2e-6
                st = r.stats()
                assert st["device_errors"] == 0
                assert st["bricks_uploaded"] + st["bricks_cached"] == st["bricks_rendered"]
                if budget == 5 and k > 0:
                    assert st["bricks_uploaded"] > 0       # streamed through the ring
                if budget == 0 and k > 0:
                    assert st["bricks_uploaded"] == 0      # every brick resident
        if mode == 0:
            ref, amb, _ = oracle_render(cube, tf, cam, brick)
            assert_parity(img, ref, amb)
        assert want.max() > 0.2     # not an empty frame


def test_two_copy_march_equals_three_on_an_orbit(vr):
    """VR_OPT_OOC_MARCH 4 on the paper's kind of camera path (an orbit about y at
    15 degrees of elevation, 30 degree field of view): no ray is dominated by y,
    so every item sweeps along the axis the three-copy march picks and the images
    are the same bit for bit, resident and streamed, with half the copies' bytes."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)
    for cam in synth.orbit((64, 64, 64), 8, 15.0, 96, 80)[::3]:
        for budget in (0, 6):
            with _ooc(vr, cube, tf, brick, budget, march=1) as r:
                r.set_camera(cam)
                want = r.render().cpu().numpy()
            with _ooc(vr, cube, tf, brick, budget, march=4) as r:
                r.set_camera(cam)
                for _ in range(2):
                    got = r.render().cpu().numpy()
                    assert np.array_equal(got, want)
                    assert r.stats()["device_errors"] == 0
        assert want[..., 3].max() > 0.05


def test_out_of_core_errors(vr, torch):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    with vr.VolumeRenderer(0) as r:
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            vr.vr_load_cube_host(r.ctx, np.zeros((1, 4, 4), np.float32))
        r.load_cube_host(cube)
        r.set_option(vr.VR_OPT_DEVICE_BUDGET, 17 ** 3 * 4)   # one brick: too small
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.brick(16, 16, 16)
        r.set_option(vr.VR_OPT_DEVICE_BUDGET, 0)
        r.brick(16, 16, 16)
        r.set_transfer_function(tf)
        r.set_camera(synth.tiny_views(width=32, height=32)[0])
        r.set_option(vr.VR_OPT_PRECISION, vr.VR_PRECISION_F16)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.render()   # reduced precision needs the texture march, which needs the cube on the device
        r.set_option(vr.VR_OPT_PRECISION, vr.VR_PRECISION_F32)
        r.render()
        # switching back to an in-core cube
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(16, 16, 16)
        r.render()
