"""CPU-only checks of the C ABI library: it loads, exports every entry point
that include/vr.h declares, rejects bad arguments, and its host-side planner
(the rendering rectangle of Section 2.3.2) never drops a pixel whose ray has a
sample in a brick (checked against the oracle's per-pixel brick ownership)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vrmod():
    from paper_1205_0282_gb300 import build
    build.build()
    from paper_1205_0282_gb300 import vr
    return vr


def _header_functions():
    text = open(os.path.join(ROOT, "include", "vr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vr_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported(vrmod):
    names = _header_functions()
    assert len(names) >= 13
    lib = vrmod._lib
    for n in names:
        assert hasattr(lib, n), f"libvr.so does not export {n}"
    assert sorted(vrmod.EXPORTS) == names


def test_header_constants_match_the_binding(vrmod):
    """Every VR_* integer constant of include/vr.h has the same value in the
    Python binding (error codes, options, kernels, precisions)."""
    text = open(os.path.join(ROOT, "include", "vr.h")).read()
    consts = {m[0]: m[1] or m[2] for m in
              re.findall(r"^#define\s+(VR_[A-Z0-9_]+)\s+(?:\((-?\d+)\)|(-?\d+))(?:\s|$)", text, flags=re.M)}
    assert len(consts) >= 21 and "VR_EINVAL" in consts and "VR_OPT_TEX_SLAB_LAYERS" in consts
    for name, value in consts.items():
        assert getattr(vrmod, name, None) == int(value), name


def test_create_without_gpu_fails_cleanly(vrmod):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(vrmod.VRError):
        vrmod.vr_create(0)


def test_null_context_calls_are_rejected(vrmod):
    lib = vrmod._lib
    assert lib.vr_brick(None, 8, 8, 8) == vrmod.VR_EINVAL
    assert lib.vr_render(None, None, None) == vrmod.VR_EINVAL
    assert lib.vr_set_option(None, 1, 1) == vrmod.VR_EINVAL
    assert lib.vr_last_error(None) == b"null context"
    lib.vr_destroy(None)


def test_plan_rects_reject_bad_arguments(vrmod):
    cam = synth.pose((64, 64, 64), 0.3, 0.2, 32, 32)
    with pytest.raises(vrmod.VRError):
        vrmod.vr_plan_brick_rects(dict(cam, width=0), (64, 64, 64), (32, 32, 32))
    with pytest.raises(vrmod.VRError):
        vrmod.vr_plan_brick_rects(dict(cam, target=cam["eye"]), (64, 64, 64), (32, 32, 32))


CASES = [
    ((64, 64, 64), (32, 32, 32), synth.tiny_views(width=96, height=80)[0]),
    ((64, 64, 64), (24, 24, 24), synth.tiny_views(width=96, height=80)[2]),
    ((61, 47, 53), (16, 20, 12), synth.pose((61, 47, 53), 2.2, -0.9, 70, 90)),
    # eye inside the cube: bricks reaching behind the eye cover the whole image
    ((64, 64, 64), (16, 16, 16), synth.camera((30, 33, 20), (60, 10, 50), (0, 1, 0), 70.0, 64, 48)),
    # wide field of view, close eye
    ((40, 40, 40), (8, 8, 8), synth.camera((19.5, 19.5, -3), (19.5, 19.5, 20), (0, 1, 0), 120.0, 50, 50)),
]


@pytest.mark.parametrize("shape,brick,cam", CASES)
def test_rendering_rectangles_are_sound(vrmod, shape, brick, cam):
    rects = vrmod.vr_plan_brick_rects(cam, shape, brick)
    W, H = cam["width"], cam["height"]
    pixels = np.arange(W * H)
    owns = oracle.pixel_bricks(cam, shape, brick, pixels)
    ii, jj = pixels % W, pixels // W
    for b in range(owns.shape[1]):
        hit = owns[:, b]
        if not hit.any():
            continue
        x0, y0, x1, y1 = rects[b]
        inside = (ii >= x0) & (ii <= x1) & (jj >= y0) & (jj <= y1)
        assert np.all(inside[hit]), f"brick {b}: pixel with samples outside its rectangle"


def test_rectangles_are_tight_enough(vrmod):
    """Rectangles are not the whole screen: the planner actually culls."""
    cam = synth.tiny_views(width=256, height=256)[0]
    rects = vrmod.vr_plan_brick_rects(cam, (64, 64, 64), (16, 16, 16))
    area = ((rects[:, 2] - rects[:, 0] + 1) * (rects[:, 3] - rects[:, 1] + 1)).mean()
    assert area < 0.1 * 256 * 256
