"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element
by element, on the same seeded inputs (tolerances in parity_util)."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


def gpu_render(vr, torch, cube, tf, cam, brick, options=None, host_out=False):
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(np.ascontiguousarray(cube)).cuda())
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        for k, v in (options or {}).items():
            r.set_option(k, v)
        if host_out:
            out = np.zeros((cam["height"], cam["width"], 4), dtype=np.float32)
            r.render(out)
            img = out
        else:
            img = r.render().cpu().numpy()
        st = r.stats()
    assert st["device_errors"] == 0, st
    return img.astype(np.float64), st


def oracle_render(cube, tf, cam, brick, mode="ea"):
    nz, ny, nx = cube.shape
    b = None if all(bb >= n - 1 for bb, n in zip(brick, (nx, ny, nz))) else brick
    return oracle.render(cube, tf, cam, brick=b, mode=mode, amb_alpha=AMB_ALPHA,
                         amb_steps=AMB_STEPS)


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_cube(), synth.tf_tiny()


@pytest.mark.parametrize("view", range(4))
def test_tiny_views_bricked(vr, torch, tiny, view):
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32))
    ref, amb, ns = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)
    assert st["samples"] >= ns.sum() > 0


@pytest.mark.parametrize("view", range(4))
def test_tiny_views_monolithic(vr, torch, tiny, view):
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, _ = gpu_render(vr, torch, cube, tf, cam, (64, 64, 64))
    ref, amb, _ = oracle_render(cube, tf, cam, (64, 64, 64))
    assert_parity(img, ref, amb)


RAGGED = [
    # shape (nx, ny, nz), brick, camera, step, tau
    ((61, 47, 53), (24, 16, 20), dict(az=2.2, el=-0.9, W=83, H=59), 0.35, 0.99),
    ((64, 64, 64), (7, 9, 11), dict(az=0.7, el=0.3, W=100, H=41), 0.5, 0.99),
    ((33, 70, 20), (32, 32, 32), dict(az=4.0, el=1.2, W=37, H=90), 1.0, 0.95),
    ((48, 40, 56), (16, 16, 16), dict(az=1.3, el=0.1, W=64, H=64), 0.25, 1.0),
]


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED)
def test_ragged_sizes(vr, torch, shape, brick, camk, step, tau):
    nx, ny, nz = shape
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick)
    ref, amb, _ = oracle_render(cube, tf, cam, brick)
    assert_parity(img, ref, amb)


def test_eye_inside_cube(vr, torch, tiny):
    cube, tf = tiny
    for cam in [synth.camera((30, 33, 20), (60, 10, 50), (0, 1, 0), 70.0, 96, 72),
                synth.camera((31.5, 31.5, 31.5), (0, 0, 0), (0, 0, 1), 90.0, 64, 64, step=0.3)]:
        img, _ = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16))
        ref, amb, _ = oracle_render(cube, tf, cam, (16, 16, 16))
        assert_parity(img, ref, amb)


def test_opaque_tf_local_termination(vr, torch, tiny):
    """Per-brick early termination active everywhere (an opaque transfer
    function): the bricked semantics must match, not the monolithic one."""
    cube, _ = tiny
    tf = synth.make_tf([0.0, 0.0, 0.3, 0.6, 0.8, 0.9, 0.95, 0.99])
    cam = synth.tiny_views(width=128, height=128)[0]
    img, _ = gpu_render(vr, torch, cube, tf, cam, (8, 8, 8))
    ref, amb, _ = oracle_render(cube, tf, cam, (8, 8, 8))
    mono, _, _ = oracle_render(cube, tf, cam, (64, 64, 64))
    assert_parity(img, ref, amb)
    assert np.abs(ref - mono).max() > 1e-3   # the two semantics really differ here


def test_nonuniform_tf(vr, torch, tiny):
    cube, _ = tiny
    tf = np.array([[-3.0, 0.0, 0.0, 1.0, 0.0], [0.8, 0.1, 0.2, 0.9, 0.0],
                   [1.1, 0.2, 0.6, 0.8, 0.01], [2.9, 0.9, 0.9, 0.9, 0.05],
                   [4.0, 1.0, 0.5, 0.1, 0.2], [9.5, 1.0, 0.0, 0.0, 0.7]])
    cam = synth.tiny_views(width=128, height=96)[1]
    img, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32))
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("kernel", ["auto", "tex", "direct"])
def test_mip_mode(vr, torch, tiny, kernel):
    """MIP + colour map (Section 2.3.3) on the texture march (the default for a cube
    within the texture limits) and on the direct march."""
    cube, tf = tiny
    cam = synth.tiny_views(width=128, height=128)[2]
    k = {"auto": vr.VR_KERNEL_AUTO, "tex": vr.VR_KERNEL_TEX, "direct": vr.VR_KERNEL_DIRECT}[kernel]
    img, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_MODE: 1, vr.VR_OPT_KERNEL: k})
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32), mode="mip")
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_mip_texture_march_ragged(vr, torch, shape, brick, camk, step, tau):
    """MIP on the texture march over ragged cubes and bricks, against the oracle."""
    cube = synth.random_cube(shape, seed=17)
    tf = synth.make_tf([0.1, 0.2, 0.4, 0.6, 0.8, 0.9, 1.0, 1.0], lo=-2.0, hi=6.0)
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick, {vr.VR_OPT_MODE: 1, vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX})
    ref, amb, _ = oracle_render(cube, tf, cam, brick, mode="mip")
    assert_parity(img, ref, amb)


def test_skip_and_cull_do_not_change_the_image(vr, torch):
    """Exact empty-space skipping (Section 2.3.1 min/max) and rendering-rectangle
    culling (Section 2.3.2) only drop work that contributes exactly zero."""
    cube = synth.hi_cube(seed=5, shape_xyz=(96, 80, 112), n_line=20, n_cont=2)
    tf = synth.tf_hi_b()
    cam = synth.pose((96, 80, 112), 0.4, 0.26, 120, 90)
    base, st = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16))
    assert st["bricks_skipped"] > 0
    noskip, st2 = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16), {vr.VR_OPT_SKIP_EMPTY: 0})
    nocull, st3 = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16), {vr.VR_OPT_RECT_CULL: 0})
    assert st2["bricks_skipped"] == 0 and st3["items"] > st["items"]
    # the dropped fragments are exactly zero; the composite's shuffle scan groups a
    # pixel's fragments in fours, so extra zero fragments can regroup the 'over'
    # products: equal up to FP32 rounding (one ulp of values <= 1)
    np.testing.assert_allclose(base, nocull, rtol=0, atol=1.2e-7)
    np.testing.assert_allclose(base, noskip, rtol=0, atol=1.2e-7)
    ref, amb, _ = oracle_render(cube, tf, cam, (16, 16, 16))
    assert_parity(base, ref, amb, min_signal=0.01)


def test_host_output_matches_device_output(vr, torch, tiny):
    cube, tf = tiny
    cam = synth.tiny_views(width=77, height=65)[3]
    dev, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32))
    host, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), host_out=True)
    np.testing.assert_array_equal(dev, host)


def test_sample_count_matches_oracle_without_termination(vr, torch, tiny):
    cube, tf = tiny
    cam = synth.tiny_views(width=96, height=96, term_alpha=1.0)[0]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32))
    ref, amb, ns = oracle_render(cube, tf, cam, (32, 32, 32))
    n_amb = int((amb != 0).sum())
    assert abs(st["samples"] - int(ns.sum())) <= n_amb
    assert_parity(img, ref, amb)


def test_brick_minmax_matches_oracle(vr, torch, tiny):
    cube, _ = tiny
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        for brick in [(32, 32, 32), (24, 16, 40), (7, 9, 11)]:
            r.brick(*brick)
            np.testing.assert_array_equal(r.brick_minmax(), oracle.brick_minmax(cube, brick))


def test_repeated_frames_and_streams(vr, torch, tiny):
    """Several frames in flight on a side stream give the same images as one
    synchronous frame each."""
    cube, tf = tiny
    views = synth.tiny_views(width=64, height=64)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        singles = []
        for cam in views:
            r.set_camera(cam)
            singles.append(r.render().cpu())
        s = torch.cuda.Stream()
        outs = []
        with torch.cuda.stream(s):
            for rep in range(3):
                for cam in views:
                    r.set_camera(cam)
                    outs.append(r.render(stream=s))
        s.synchronize()
        for k, o in enumerate(outs):
            assert torch.equal(o.cpu(), singles[k % 4])
        assert r.stats()["frames"] == 16


def test_error_codes(vr, torch, tiny):
    cube, tf = tiny
    r = vr.VolumeRenderer(0)
    out = torch.empty((8, 8, 4), device="cuda")
    with pytest.raises(vr.VRError) as e:
        r.render(out)
    assert e.value.code == vr.VR_ESTATE
    with pytest.raises(vr.VRError) as e:
        r.brick(8, 8, 8)
    assert e.value.code == vr.VR_ESTATE
    r.load_cube(torch.from_numpy(cube).cuda())
    with pytest.raises(vr.VRError) as e:
        r.brick(0, 8, 8)
    assert e.value.code == vr.VR_EINVAL
    bad = tf.copy()
    bad[3, 0] = bad[2, 0]
    with pytest.raises(vr.VRError) as e:
        r.set_transfer_function(bad)
    assert e.value.code == vr.VR_EINVAL
    with pytest.raises(vr.VRError) as e:
        r.set_camera(synth.camera((0, 0, 0), (0, 0, 0), (0, 1, 0)))
    assert e.value.code == vr.VR_EINVAL
    with pytest.raises(vr.VRError) as e:
        r.set_option(99, 1)
    assert e.value.code == vr.VR_EINVAL
    r.close()


@pytest.mark.parametrize("view", [0, 3])
def test_direct_gather_kernel(vr, torch, tiny, view):
    """The L1-gather march (8x8 items) against the oracle, for the A/B comparison
    with the TMA-staged march."""
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_KERNEL: vr.VR_KERNEL_DIRECT})
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)
    assert st["chunks_staged"] == 0


@pytest.mark.parametrize("view", range(4))
def test_tma_kernel_stages_chunks(vr, torch, tiny, view):
    """The TMA-staged march (16x16 items, boxes copied into shared memory)."""
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TMA})
    assert st["chunks_staged"] > 0
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)


def test_tma_fallback_chunks(vr, torch, tiny):
    """A coarse image (several voxels per pixel) gives chunk footprints larger than
    the staged box; those chunks read through L1 and the image still matches."""
    cube, tf = tiny
    cam = synth.tiny_views(width=20, height=18)[0]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TMA})
    assert st["chunks_direct"] > 0
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)


def test_kernels_agree(vr, torch):
    cube = synth.hi_cube(seed=9, shape_xyz=(128, 96, 160), n_line=40, n_cont=3)
    tf = synth.tf_hi_a()
    for az in (0.3, 1.6, 3.9):
        cam = synth.pose((128, 96, 160), az, 0.26, 160, 120)
        a, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32))
        for k in (vr.VR_KERNEL_DIRECT, vr.VR_KERNEL_TMA, vr.VR_KERNEL_TEX):
            b, _ = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_KERNEL: k})
            assert np.abs(a - b).max() < 1e-4
        ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
        assert_parity(a, ref, amb)


@pytest.mark.parametrize("view", [0, 1, 2, 3])
def test_texture_gather_kernel(vr, torch, tiny, view):
    """The texture-gather march (unfiltered tld4 gathers from layered textures,
    FP32 trilinear weights) against the oracle."""
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX})
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_texture_gather_ragged(vr, torch, shape, brick, camk, step, tau):
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick, {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX})
    ref, amb, _ = oracle_render(cube, tf, cam, brick)
    assert_parity(img, ref, amb)


def test_mip_stops_at_the_global_maximum(vr, torch):
    """Section 2.3.2: a MIP ray stops once it reaches the cube's global maximum.
    On a cube clipped low (large plateaus at the maximum) the
    image is unchanged and fewer samples are taken than the oracle's full rays."""
    cube = synth.tiny_cube()
    # clipped at its 30th percentile: 70% of the voxels sit at the maximum, so many
    # cells have all eight corners there and a ray soon samples the maximum exactly
    cube = np.minimum(cube, np.percentile(cube, 30)).astype(np.float32)
    tf = synth.make_tf([0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8], lo=float(cube.min()), hi=float(cube.max()))
    cam = synth.tiny_views(width=96, height=96)[1]
    ref, amb, ns = oracle_render(cube, tf, cam, (32, 32, 32), mode="mip")
    for kernel in (vr.VR_KERNEL_TEX, vr.VR_KERNEL_DIRECT):
        img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_MODE: 1, vr.VR_OPT_KERNEL: kernel})
        assert_parity(img, ref, amb, min_signal=0.0)
        assert st["samples"] < 0.7 * ns.sum()


# ------------------------------------------------------------------ dynamic step

@pytest.mark.parametrize("view", range(4))
def test_dynamic_step_texture_march(vr, torch, tiny, view):
    """Section 2.3.2's dynamic step (samples `step` voxels apart along each ray's
    dominant axis) on the default texture march, against the oracle."""
    cube, tf = tiny
    cam = synth.tiny_views()[view]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_STEP_MODE: 1})
    ref, amb, ns = oracle.render(cube, tf, cam, brick=(32, 32, 32), amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS,
                                 step_mode=1)
    assert_parity(img, ref, amb)
    fixed, _, nf = oracle.render(cube, tf, cam, brick=(32, 32, 32))
    assert np.abs(ref - fixed).max() > 1e-3      # the variant does change the image


@pytest.mark.parametrize("kernel,mode", [(1, 0), (1, 1), (2, 1)])
def test_dynamic_step_direct_march_and_mip(vr, torch, tiny, kernel, mode):
    cube, tf = tiny
    cam = synth.tiny_views(width=120, height=100)[2]
    img, _ = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16),
                        {vr.VR_OPT_STEP_MODE: 1, vr.VR_OPT_KERNEL: kernel, vr.VR_OPT_MODE: mode})
    ref, amb, _ = oracle.render(cube, tf, cam, brick=(16, 16, 16), mode="mip" if mode else "ea",
                                amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS, step_mode=1)
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_dynamic_step_ragged(vr, torch, shape, brick, camk, step, tau):
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick, {vr.VR_OPT_STEP_MODE: 1})
    ref, amb, _ = oracle.render(cube, tf, cam, brick=brick, amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS, step_mode=1)
    assert_parity(img, ref, amb)


def test_dynamic_step_errors(vr, torch, tiny):
    cube, tf = tiny
    cam = synth.tiny_views(width=32, height=32)[0]
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.set_option(vr.VR_OPT_STEP_MODE, 2)
        r.set_option(vr.VR_OPT_STEP_MODE, 1)
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TMA)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.render()
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_AUTO)
        r.render()
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            vr.Server(r, 128 << 20)


def test_asynchronous_host_output():
    """VR_OPT_HOST_OUTPUT_ASYNC: frames rendered into page-locked host buffers
    without waiting (several in flight) hold the synchronous images once the
    stream is synchronised; pageable memory is refused."""
    import torch
    from paper_1205_0282_gb300 import vr
    cube = synth.tiny_cube()
    tf = synth.tf_tiny()
    cams = synth.tiny_views(width=120, height=90)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        want = []
        for cam in cams:
            r.set_camera(cam)
            want.append(r.render(np.zeros((90, 120, 4), np.float32)).copy())
        r.set_option(vr.VR_OPT_HOST_OUTPUT_ASYNC, 1)
        bufs = [torch.full((90, 120, 4), -1.0, pin_memory=True).numpy() for _ in cams]
        for cam, b in zip(cams, bufs):
            r.set_camera(cam)
            r.render(b)
        torch.cuda.synchronize()
        for b, w in zip(bufs, want):
            assert np.array_equal(b, w)
        assert want[0][..., 3].max() > 0.1
        with pytest.raises(vr.VRError) as e:
            r.render(np.zeros((90, 120, 4), np.float32))
        assert e.value.code == vr.VR_EINVAL


def test_camera_from_opengl_matrices_renders_the_same_image():
    """vr_set_camera_matrices with the viewer's modelview and projection (the
    paper's interface) renders the image of the equivalent look-at camera, and
    the oracle's."""
    import torch
    from paper_1205_0282_gb300 import vr
    from test_abi_host import _look_at, _perspective
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views(width=120, height=90)[1]
    view = _look_at(cam["eye"], cam["target"], cam["up"])
    proj = _perspective(cam["fovy_deg"], 120 / 90)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        want = r.render().cpu().numpy().astype(np.float64)
        r.set_camera_matrices(view, proj, 120, 90, cam["step"], cam["term_alpha"])
        got = r.render().cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= 1e-6
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(got, ref, amb)
