"""GPU tests of the brick-provider load (vr_load_cube_provider): a cube that
exists only as a function (the seeded generator's native block source, or a
Python callable) renders exactly like the same cube held in host memory
(vr_load_cube_host), with every brick resident and streamed through a small
cache, on both out-of-core marches; the bricks' ranges are the host store's;
a provider that fails makes vr_brick and vr_render return VR_ESOURCE, and a
frame that failed renders correctly once the provider answers again.  The
learned context's fallback takes its plain blocks from a provider with the same
errors and images as from the host cube.  Every failure here happens on the
host (the provider returns an error code): no kernel is made to fail."""
import threading

import numpy as np
import pytest

import oracle
import synth
from ooc_budget import budget_for
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity

pytestmark = pytest.mark.gpu

SHAPE = (61, 47, 53)          # ragged: no brick size below divides n - 1
SEED, N_LINE, N_CONT = 11, 14, 2


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


@pytest.fixture(scope="module")
def source():
    return synth.BlockSource(SHAPE, SEED, synth.hi_sources(SEED, SHAPE, N_LINE, N_CONT))


@pytest.fixture(scope="module")
def cube():
    return synth.hi_cube(seed=SEED, shape_xyz=SHAPE, n_line=N_LINE, n_cont=N_CONT)


def _ctx(vr, load, brick, tf, cam, march, budget_bricks=0):
    r = vr.VolumeRenderer(0)
    load(r)
    r.set_option(vr.VR_OPT_OOC_MARCH, march)
    if budget_bricks:
        r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget_for(budget_bricks, brick, march))
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_camera(cam)
    return r


def test_native_block_source_equals_the_whole_cube(source, cube):
    """The generator's blocks are the whole cube's voxels bit for bit (the
    provider's layout: row and slice strides in floats)."""
    for origin, extent in [((0, 0, 0), SHAPE), ((13, 5, 40), (17, 17, 13)), ((60, 46, 52), (1, 1, 1))]:
        blk = source.block(origin, extent)
        x, y, z = origin
        ex, ey, ez = extent
        assert np.array_equal(blk.view(np.uint32), cube[z:z + ez, y:y + ey, x:x + ex].view(np.uint32))


@pytest.mark.parametrize("march", [1, 0])
@pytest.mark.parametrize("budget", [0, 5])
def test_provider_renders_the_host_cube_image(vr, source, cube, march, budget):
    brick = (16, 16, 16)          # 4 x 3 x 4 bricks, the last ones partial
    tf = synth.tf_tiny()
    cams = [synth.pose(SHAPE, a, e, 96, 72) for a, e in ((0.4, 0.3), (2.5, -0.6))]
    host = _ctx(vr, lambda r: r.load_cube_host(cube), brick, tf, cams[0], march, budget)
    prov = _ctx(vr, lambda r: r.load_cube_provider(source, SHAPE), brick, tf, cams[0], march, budget)
    assert np.array_equal(prov.brick_minmax(), host.brick_minmax())
    for k in range(4):
        cam = cams[k % 2]
        host.set_camera(cam)
        prov.set_camera(cam)
        prov.reset_stats()
        want = host.render().cpu().numpy()
        got = prov.render().cpu().numpy()
        assert np.array_equal(got, want)
        st = prov.stats()
        assert st["device_errors"] == 0
        assert st["bricks_uploaded"] + st["bricks_cached"] == st["bricks_rendered"]
        if budget and k > 0:
            assert st["bricks_uploaded"] > 0     # streamed frame after frame
        if not budget and k > 1:
            assert st["bricks_uploaded"] == 0    # every brick stays resident
    host.close()
    prov.close()


def test_provider_matches_the_oracle(vr, source, cube):
    brick = (24, 16, 20)
    tf = synth.tf_tiny()
    cam = synth.pose(SHAPE, 2.2, -0.9, 83, 59, step=0.35, term_alpha=0.99)
    with _ctx(vr, lambda r: r.load_cube_provider(source, SHAPE), brick, tf, cam, 1, 4) as r:
        got = r.render().cpu().numpy().astype(np.float64)
    want, amb, _ = oracle.render(cube, tf, cam, brick=brick, amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert want[..., 3].max() > 0.05
    assert_parity(got, want, amb)


def test_python_callable_provider(vr, cube):
    """A Python callable serves as the provider (called from the library's host
    threads); its blocks are asked for inside the cube only."""
    calls = []
    lock = threading.Lock()

    def provide(origin, extent):
        x, y, z = origin
        ex, ey, ez = extent
        assert min(origin) >= 0 and x + ex <= SHAPE[0] and y + ey <= SHAPE[1] and z + ez <= SHAPE[2]
        with lock:
            calls.append((origin, extent))
        return cube[z:z + ez, y:y + ey, x:x + ex]

    brick = (32, 32, 32)          # 2 x 2 x 2 bricks
    tf = synth.tf_tiny()
    cam = synth.pose(SHAPE, 1.1, 0.2, 64, 48)
    with _ctx(vr, lambda r: r.load_cube_host(cube), brick, tf, cam, 1) as r:
        want = r.render().cpu().numpy()
    with _ctx(vr, lambda r: r.load_cube_provider(provide, SHAPE), brick, tf, cam, 1) as r:
        assert len(calls) == 8        # vr_brick: every brick once, for its range
        r.set_option(vr.VR_OPT_PROVIDER_THREADS, 2)
        got = r.render().cpu().numpy()
    assert np.array_equal(got, want)
    assert (((32, 0, 0), (29, 33, 33))) in calls   # the last brick along x: 61 - 32 voxels with the apron


def test_failing_provider(vr, cube):
    """A provider failure is reported as VR_ESOURCE by vr_brick and by vr_render;
    the failed frame's bricks are asked for again by the next frame, which then
    renders the right image."""
    state = {"fail_from": 10 ** 9, "calls": 0}
    lock = threading.Lock()

    def provide(origin, extent):
        with lock:
            state["calls"] += 1
            if state["calls"] > state["fail_from"]:
                raise RuntimeError("storage unavailable")
        x, y, z = origin
        ex, ey, ez = extent
        return cube[z:z + ez, y:y + ey, x:x + ex]

    brick = (16, 16, 16)
    tf = synth.tf_tiny()
    cam = synth.pose(SHAPE, 0.4, 0.3, 80, 64)
    with _ctx(vr, lambda r: r.load_cube_host(cube), brick, tf, cam, 1) as r:
        want = r.render().cpu().numpy()
    r = vr.VolumeRenderer(0)
    r.load_cube_provider(provide, SHAPE)
    state["fail_from"] = 20
    with pytest.raises(vr.VRError) as e:
        r.brick(*brick)
    assert e.value.code == vr.VR_ESOURCE and "brick" in vr.vr_last_error(r.ctx)
    state["fail_from"] = 10 ** 9
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_camera(cam)
    state["calls"], state["fail_from"] = 0, 3      # the frame's uploads fail part-way
    with pytest.raises(vr.VRError) as e:
        r.render()
    assert e.value.code == vr.VR_ESOURCE
    state["fail_from"] = 10 ** 9
    for _ in range(2):
        assert np.array_equal(r.render().cpu().numpy(), want)
    r.close()


def test_learned_fallback_from_a_provider(vr):
    """The fallback scan and the fallback bricks' plain blocks from a provider:
    the same per-brick errors and the same image as from the host cube."""
    import torch
    from test_gpu_codec import _ctx as codec_ctx, _fallback_case
    cube, shape, brick, c, tf, cam = _fallback_case(vr, torch)

    def provide(origin, extent):
        x, y, z = origin
        ex, ey, ez = extent
        return cube[z:z + ez, y:y + ey, x:x + ex]

    with codec_ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=float("inf")) as r:
        err, _ = r.codec_brick_errors()
    bound = float(np.median(err))
    for budget in (0, 3):
        with codec_ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=bound, budget=budget) as r:
            want_err, want_n = r.codec_brick_errors()
            want = r.render().cpu().numpy()
        r = vr.VolumeRenderer(0)
        r.load_cube_codec(c, shape)
        r.set_codec_fallback_provider(provide, bound)
        r.set_option(vr.VR_OPT_OOC_MARCH, 1)      # as the host-cube context: the texture march
        if budget:
            r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget_for(budget, brick, 1))
        r.set_option(vr.VR_OPT_SKIP_EMPTY, 0)
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        got_err, got_n = r.codec_brick_errors()
        got = r.render().cpu().numpy()
        r.close()
        assert np.array_equal(got_err, want_err) and got_n == want_n and 0 < got_n < 12
        assert np.array_equal(got, want)
    c.close()


@pytest.mark.parametrize("march", [1, 3, 0])
def test_provider_mip_and_dynamic_step(vr, source, cube, march):
    """MIP with the dynamic step through a provider-backed cache (every march
    of the out-of-core path): the host-cube context's image bit for bit, and the
    oracle's."""
    brick = (24, 16, 20)
    tf = synth.tf_tiny()
    cam = synth.pose(SHAPE, 0.7, 0.4, 90, 70, step=0.4)

    def ctx(load):
        r = vr.VolumeRenderer(0)
        load(r)
        r.set_option(vr.VR_OPT_OOC_MARCH, march)
        r.set_option(vr.VR_OPT_MODE, 1)
        r.set_option(vr.VR_OPT_STEP_MODE, 1)
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        return r

    with ctx(lambda r: r.load_cube_host(cube)) as r:
        want = r.render().cpu().numpy()
    with ctx(lambda r: r.load_cube_provider(source, SHAPE)) as r:
        got = r.render().cpu().numpy()
    assert np.array_equal(got, want) and got.max() > 0.2
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, mode="mip", amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS,
                                step_mode=1)
    assert_parity(got.astype(np.float64), ref, amb)

