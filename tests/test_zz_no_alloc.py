"""The allocation-free entry point (vr_render_noalloc) renders the same images
as vr_render, and the images of the FP64 oracle.

vr_render_noalloc is for callers that may not allocate device memory while
rendering (an application that owns the device-memory budget, a real-time loop
that cannot take cudaMalloc's implicit synchronisation, an embedding with its
own allocator): its scratch lives in a static device array inside the library.
This file is collected last so that, in a run that stops at the first failure,
every other test has already run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, MAX_TOL, RMS_TOL, assert_parity

pytestmark = pytest.mark.gpu


def _reference(vr, dcube, brick, tf, cams):
    """vr_render's images of the same frames (context path)."""
    refs = []
    with vr.VolumeRenderer(0) as r:
        r.load_cube(dcube)
        r.brick(*brick)
        r.set_transfer_function(tf)
        for cam in cams:
            r.set_camera(cam)
            refs.append(r.render().cpu().numpy().astype(np.float64))
    return refs


def _close(got, ref):
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    assert err.max() <= MAX_TOL and np.sqrt(np.mean(err ** 2)) <= RMS_TOL, err.max()


def test_noalloc_matches_vr_render_on_two_calls_in_a_row():
    import torch
    from paper_1205_0282_gb300 import vr

    cube = synth.tiny_cube()
    tf = synth.tf_tiny()
    cams = synth.tiny_views(width=200, height=150)[:2]
    dcube = torch.from_numpy(cube).cuda()
    refs = _reference(vr, dcube, (32, 32, 32), tf, cams)
    for cam, ref in zip(cams, refs):          # two calls in a row, sharing the scratch
        out = torch.full((cam["height"], cam["width"], 4), -1.0, device="cuda")
        vr.vr_render_noalloc(dcube, (32, 32, 32), tf, cam, out)
        torch.cuda.synchronize()
        assert ref[..., 3].max() > 0.1
        _close(out.cpu().numpy(), ref)


def test_noalloc_back_to_back_calls_keep_their_own_plans():
    """Three calls enqueued on one stream without waiting in between: each
    fills a host staging set while earlier uploads may still be pending, and
    each frame still gets its own plan."""
    import torch
    from paper_1205_0282_gb300 import vr

    cube = synth.tiny_cube()
    tf = synth.tf_tiny()
    cams = synth.tiny_views(width=160, height=120)[:3]
    dcube = torch.from_numpy(cube).cuda()
    refs = _reference(vr, dcube, (16, 16, 16), tf, cams)
    outs = [torch.full((c["height"], c["width"], 4), -1.0, device="cuda") for c in cams]
    for cam, out in zip(cams, outs):   # each frame's image goes to its own buffer; the
        vr.vr_render_noalloc(dcube, (16, 16, 16), tf, cam, out)   # shared scratch is stream-ordered
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        _close(out.cpu().numpy(), ref)


CASES = [
    # (name, cube, brick, tf, camera)
    ("eye inside the cube", "tiny", (16, 16, 16), "tiny",
     synth.camera((30, 33, 20), (60, 10, 50), (0, 1, 0), 70.0, 96, 72)),
    ("non-uniform transfer function", "tiny", (32, 32, 32), "nonuniform", synth.tiny_views(width=128, height=96)[1]),
    ("ragged cube and bricks", "ragged", (24, 16, 20), "tiny",
     synth.pose((61, 47, 53), 2.2, -0.9, 83, 59, step=0.35, term_alpha=0.99)),
]
NONUNIFORM = np.array([[-3.0, 0.0, 0.0, 1.0, 0.0], [0.8, 0.1, 0.2, 0.9, 0.0],
                       [1.1, 0.2, 0.6, 0.8, 0.01], [2.9, 0.9, 0.9, 0.9, 0.05],
                       [4.0, 1.0, 0.5, 0.1, 0.2], [9.5, 1.0, 0.0, 0.0, 0.7]])


@pytest.mark.parametrize("name,cube_kind,brick,tf_kind,cam", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_vr_render_and_the_oracle(name, cube_kind, brick, tf_kind, cam):
    import torch
    from paper_1205_0282_gb300 import vr

    cube = synth.tiny_cube() if cube_kind == "tiny" else synth.hi_cube(seed=11, shape_xyz=(61, 47, 53),
                                                                        n_line=12, n_cont=2)
    tf = synth.tf_tiny() if tf_kind == "tiny" else NONUNIFORM
    dcube = torch.from_numpy(cube).cuda()
    ref = _reference(vr, dcube, brick, tf, [cam])[0]
    out = torch.full((cam["height"], cam["width"], 4), -1.0, device="cuda")
    vr.vr_render_noalloc(dcube, brick, tf, cam, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    _close(got, ref)
    want, amb, _ = oracle.render(cube, tf, cam, brick=brick, amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert_parity(got, want, amb)


def test_noalloc_rejects_frames_beyond_its_limits():
    """Every rejection below happens on the host: no kernel is launched."""
    import torch
    from paper_1205_0282_gb300 import vr

    cube = torch.from_numpy(synth.tiny_cube()).cuda()
    tf = synth.tf_tiny()
    too_wide = synth.tiny_views(width=2048, height=64)[0]
    out = torch.empty((64, 2048, 4), device="cuda")
    with pytest.raises(vr.VRError) as e:
        vr.vr_render_noalloc(cube, (32, 32, 32), tf, too_wide, out)
    assert e.value.code == vr.VR_EINVAL
    cam = synth.tiny_views(width=64, height=64)[0]
    with pytest.raises(ValueError):           # host image
        vr.vr_render_noalloc(cube, (32, 32, 32), tf, cam, np.zeros((64, 64, 4), dtype=np.float32))
    with pytest.raises(ValueError):           # image smaller than the frame
        vr.vr_render_noalloc(cube, (32, 32, 32), tf, cam, torch.empty((32, 64, 4), device="cuda"))
    with pytest.raises(ValueError):           # FP16 cube
        vr.vr_render_noalloc(cube.half(), (32, 32, 32), tf, cam, torch.empty((64, 64, 4), device="cuda"))
    with pytest.raises(ValueError):           # FP64 image
        vr.vr_render_noalloc(cube, (32, 32, 32), tf, cam,
                             torch.empty((64, 64, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):           # host cube
        vr.vr_render_noalloc(cube.cpu(), (32, 32, 32), tf, cam, torch.empty((64, 64, 4), device="cuda"))
