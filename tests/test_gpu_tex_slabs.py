"""Texture march with its layered copies split into slabs along their layer axis.

A slab holds whole bricks plus the next brick's first layer (the apron), so every
sample reads the same texels as from one unsplit copy: the images must agree
bit for bit, in every storage, and with the FP64 oracle.  Small slab limits
(VR_OPT_TEX_SLAB_LAYERS) make small cubes exercise several slabs per axis.
"""
import numpy as np
import pytest

import synth
from parity_util import assert_parity
from test_gpu_render import RAGGED, gpu_render, oracle_render, torch  # noqa: F401  (torch: fixture)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


@pytest.mark.parametrize("precision", ["f32", "f16", "f8"])
@pytest.mark.parametrize("view", range(4))
def test_slabs_match_one_copy(vr, torch, precision, view):
    """Bricks of 16 in a 64^3 cube; slabs of 2 bricks (33 layers) or of 1 brick (17
    layers) along every axis give the image of the unsplit copies exactly."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views()[view]
    prec = {"f32": vr.VR_PRECISION_F32, "f16": vr.VR_PRECISION_F16, "f8": vr.VR_PRECISION_F8}[precision]
    base = {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX, vr.VR_OPT_PRECISION: prec}
    ref, st0 = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16), base)
    for layers in (33, 17):
        img, st = gpu_render(vr, torch, cube, tf, cam, (16, 16, 16), {**base, vr.VR_OPT_TEX_SLAB_LAYERS: layers})
        assert np.array_equal(img, ref), (layers, np.abs(img - ref).max())
        assert st["samples"] == st0["samples"]


@pytest.mark.parametrize("shape,brick,camk,step,tau", RAGGED[:2])
def test_slabs_ragged_against_oracle(vr, torch, shape, brick, camk, step, tau):
    """Ragged cubes and bricks (the last slab and the last brick partial), one
    brick per slab, against the FP64 oracle; MIP too."""
    cube = synth.random_cube(shape, seed=23)
    tf = synth.make_tf([0, 0.01, 0.02, 0.05, 0.1, 0.2, 0.3, 0.5], lo=-2.0, hi=6.0)
    cam = synth.pose(shape, camk["az"], camk["el"], camk["W"], camk["H"], step=step, term_alpha=tau)
    opts = {vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX, vr.VR_OPT_TEX_SLAB_LAYERS: max(brick) + 1}
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick, opts)
    ref, amb, _ = oracle_render(cube, tf, cam, brick)
    assert_parity(img, ref, amb)
    img, _ = gpu_render(vr, torch, cube, tf, cam, brick, {**opts, vr.VR_OPT_MODE: 1})
    ref, amb, _ = oracle_render(cube, tf, cam, brick, mode="mip")
    assert_parity(img, ref, amb)


def test_slab_limit_below_one_brick(vr, torch):
    """A slab limit below one brick plus its apron leaves no texture march: the
    automatic choice falls back to the TMA march (oracle parity), an explicit
    texture request fails with VR_EINVAL, a negative limit is rejected."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    cam = synth.tiny_views()[0]
    img, st = gpu_render(vr, torch, cube, tf, cam, (32, 32, 32), {vr.VR_OPT_TEX_SLAB_LAYERS: 32})
    assert st["chunks_staged"] + st["chunks_direct"] > 0      # the TMA march ran
    ref, amb, _ = oracle_render(cube, tf, cam, (32, 32, 32))
    assert_parity(img, ref, amb)
    with pytest.raises(vr.VRError, match="VR_EINVAL"):
        gpu_render(vr, torch, cube, tf, cam, (32, 32, 32),
                   {vr.VR_OPT_TEX_SLAB_LAYERS: 32, vr.VR_OPT_KERNEL: vr.VR_KERNEL_TEX})
    with vr.VolumeRenderer(0) as r:
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.set_option(vr.VR_OPT_TEX_SLAB_LAYERS, -1)
