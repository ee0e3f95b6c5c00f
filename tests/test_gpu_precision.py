"""GPU parity of the reduced-precision storage forms (VR_OPT_PRECISION) of the
texture-gather march.

An FP16 or FP8 render is defined as the FP32 render of the cube of values that the
storage reads back (oracle/quant.py builds that cube from the format definitions);
so each form is compared element by element with the FP64 oracle run on the
read-back cube, at the same tolerances as the FP32 path.  Cubes whose values the
storage holds exactly must give the FP32 image (FP16: bit for bit; FP8, which
interpolates code values and applies the brick's scale once afterwards: up to
FP32 rounding).  This checks the code layout, the decode and the per-brick scale
of every corner, including the corners a brick reads from its neighbours.
"""
import numpy as np
import pytest

import synth
from oracle import quant
from parity_util import assert_parity
from test_gpu_render import RAGGED, gpu_render, oracle_render
from test_oracle_pins import fp8_lossless_cube

pytestmark = pytest.mark.gpu

PREC = {"f16": 1, "f8": 2}


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


def tex_render(vr, torch, cube, tf, cam, brick, prec, extra=None):
    opts = {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX, vr.VR_OPT_PRECISION: PREC.get(prec, 0)}
    opts.update(extra or {})
    return gpu_render(vr, torch, cube, tf, cam, brick, opts)


@pytest.mark.parametrize("prec", ["f16", "f8"])
@pytest.mark.parametrize("view", range(4))
def test_tiny_views(vr, torch, prec, view):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (32, 32, 32)
    cam = synth.tiny_views()[view]
    img, st = tex_render(vr, torch, cube, tf, cam, brick, prec)
    ref, amb, _ = oracle_render(quant.stored_cube(cube, prec, brick), tf, cam, brick)
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("prec", ["f16", "f8"])
@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_ragged(vr, torch, prec, shape, brick, camk, step, tau):
    cube = synth.hi_cube(seed=11, shape_xyz=shape, n_line=12, n_cont=2)
    tf = synth.tf_tiny()
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    img, _ = tex_render(vr, torch, cube, tf, cam, brick, prec)
    ref, amb, _ = oracle_render(quant.stored_cube(cube, prec, brick), tf, cam, brick)
    assert_parity(img, ref, amb)


@pytest.mark.parametrize("shape,brick", [((40, 33, 27), (16, 16, 8)), ((64, 64, 64), (32, 32, 32)),
                                         ((61, 47, 53), (24, 16, 20))])
def test_fp8_exact_cube_gives_the_fp32_image(vr, torch, shape, brick):
    cube = fp8_lossless_cube(shape, brick)
    assert np.array_equal(quant.stored_cube(cube, "f8", brick), cube)
    tf = synth.make_tf([0.0, 0.02, 0.05, 0.08, 0.12, 0.2, 0.3, 0.4], lo=-3.0, hi=14.0)
    for az, el in [(0.4, 0.3), (2.1, -0.7), (4.4, 1.1)]:
        cam = synth.pose(shape, az, el, 96, 80, step=0.4)
        a, _ = tex_render(vr, torch, cube, tf, cam, brick, "f32")
        b, _ = tex_render(vr, torch, cube, tf, cam, brick, "f8")
        assert np.abs(a - b).max() <= 2e-6
        assert np.mean(a == b) > 0.9
        assert a[..., 3].max() > 0.3


def test_fp16_exact_cube_gives_the_fp32_image(vr, torch):
    shape, brick = (61, 47, 53), (24, 16, 20)
    cube = quant.stored_cube(synth.hi_cube(seed=4, shape_xyz=shape, n_line=12, n_cont=2), "f16")
    tf = synth.tf_tiny()
    for az, el in [(0.4, 0.3), (2.1, -0.7)]:
        cam = synth.pose(shape, az, el, 96, 80, step=0.4)
        a, _ = tex_render(vr, torch, cube, tf, cam, brick, "f32")
        b, _ = tex_render(vr, torch, cube, tf, cam, brick, "f16")
        assert np.array_equal(a, b)


def test_skipping_uses_the_stored_range(vr, torch):
    """Empty-space skipping with reduced-precision storage is exact for the stored
    values: skipping on or off gives the same image."""
    shape, brick = (64, 64, 64), (16, 16, 16)
    cube = synth.tiny_cube()
    tf = synth.tf_hi_b()
    cam = synth.pose(shape, 0.9, 0.4, 120, 100)
    for prec in ("f16", "f8"):
        a, sa = tex_render(vr, torch, cube, tf, cam, brick, prec)
        b, _ = tex_render(vr, torch, cube, tf, cam, brick, prec, {vr.VR_OPT_SKIP_EMPTY: 0})
        assert sa["bricks_skipped"] > 0
        assert np.abs(a - b).max() < 1e-6


def test_touched_bytes_follow_the_storage(vr, torch):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views()[0]
    t = {}
    for prec in ("f32", "f16", "f8"):
        _, st = tex_render(vr, torch, cube, tf, cam, (32, 32, 32), prec)
        t[prec] = st["touched_bytes"]
    assert t["f32"] == 2 * t["f16"] == 4 * t["f8"] > 0


def test_switching_precision_and_rebricking(vr, torch):
    """One renderer switching storage and bricking gives the images of fresh ones."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views()[1]
    fresh = {}
    for prec, brick in [("f8", (32, 32, 32)), ("f32", (32, 32, 32)), ("f16", (32, 32, 32)),
                        ("f8", (16, 24, 20))]:
        fresh[prec, brick], _ = tex_render(vr, torch, cube, tf, cam, brick, prec)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.set_transfer_function(tf)
        r.set_camera(cam)
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TEX)
        for prec, brick in [("f8", (32, 32, 32)), ("f32", (32, 32, 32)), ("f16", (32, 32, 32)),
                            ("f8", (32, 32, 32)), ("f8", (16, 24, 20))]:
            r.brick(*brick)
            r.set_option(vr.VR_OPT_PRECISION, PREC.get(prec, 0))
            img = r.render().cpu().numpy().astype(np.float64)
            assert np.array_equal(img, fresh[prec, brick]), (prec, brick)


def test_precision_errors(vr, torch):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views()[0]
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.set_option(vr.VR_OPT_PRECISION, 3)
        r.set_option(vr.VR_OPT_PRECISION, vr.VR_PRECISION_F8)
        for k in (vr.VR_KERNEL_TMA, vr.VR_KERNEL_DIRECT):
            r.set_option(vr.VR_OPT_KERNEL, k)
            with pytest.raises(vr.VRError, match="VR_EINVAL"):
                r.render()
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_AUTO)
        r.set_option(vr.VR_OPT_MODE, 1)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.render()
        r.set_option(vr.VR_OPT_MODE, 0)
        r.render()  # AUTO picks the texture march for this cube
        big = cube.copy()
        big[3, 4, 5] = 70000.0
        r.load_cube(torch.from_numpy(big).cuda())
        r.brick(32, 32, 32)
        r.set_option(vr.VR_OPT_PRECISION, vr.VR_PRECISION_F16)
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.render()
        r.set_option(vr.VR_OPT_PRECISION, vr.VR_PRECISION_F8)
        r.render()
