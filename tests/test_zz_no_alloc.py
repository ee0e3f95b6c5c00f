"""The allocation-free entry point (vr_render_noalloc) renders the same images
as vr_render.

vr_render_noalloc is for callers that may not allocate device memory while
rendering (an application that owns the device-memory budget, a real-time loop
that cannot take cudaMalloc's implicit synchronisation, an embedding with its
own allocator): its scratch lives in a static device array inside the library.
This file is collected last so that, in a run that stops at the first failure,
every other test has already run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from parity_util import MAX_TOL, RMS_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_vr_render_on_two_calls_in_a_row():
    import torch
    from paper_1205_0282_gb300 import vr

    cube = synth.tiny_cube()
    tf = synth.tf_tiny()
    cams = synth.tiny_views(width=200, height=150)[:2]
    dcube = torch.from_numpy(cube).cuda()
    with vr.VolumeRenderer(0) as r:
        r.load_cube(dcube)
        r.brick(32, 32, 32)
        r.set_transfer_function(tf)
        refs = []
        for cam in cams:
            r.set_camera(cam)
            refs.append(r.render().cpu().numpy().astype(np.float64))
    for cam, ref in zip(cams, refs):          # two calls in a row, sharing the scratch
        out = torch.full((cam["height"], cam["width"], 4), -1.0, device="cuda")
        vr.vr_render_noalloc(dcube, (32, 32, 32), tf, cam, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        assert ref[..., 3].max() > 0.1
        assert err.max() <= MAX_TOL and np.sqrt(np.mean(err ** 2)) <= RMS_TOL, err.max()


def test_noalloc_rejects_frames_beyond_its_limits():
    import torch
    from paper_1205_0282_gb300 import vr

    cube = torch.from_numpy(synth.tiny_cube()).cuda()
    too_wide = synth.tiny_views(width=2048, height=64)[0]
    out = torch.empty((64, 2048, 4), device="cuda")
    with pytest.raises(vr.VRError) as e:
        vr.vr_render_noalloc(cube, (32, 32, 32), synth.tf_tiny(), too_wide, out)
    assert e.value.code == vr.VR_EINVAL
    host_out = np.zeros((64, 64, 4), dtype=np.float32)
    with pytest.raises(vr.VRError):
        vr.vr_render_noalloc(cube, (32, 32, 32), synth.tf_tiny(),
                             synth.tiny_views(width=64, height=64)[0], host_out)
