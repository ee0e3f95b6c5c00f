"""Parity at the benchmark's full size and launch configuration: the 1024 x
1024 x 2048 HI-survey cube, 128^3 bricks, 1920 x 1080 frames of the orbit the
benchmark times.  The oracle recomputes a sample of pixels one by one (random
pixels plus a dense crop) and the GPU frame must match it there."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    import torch
    from paper_1205_0282_gb300 import VolumeRenderer
    cube = synth.hi_cube()
    r = VolumeRenderer(0)
    d = torch.from_numpy(cube).cuda()
    r.load_cube(d)
    del d
    torch.cuda.empty_cache()
    r.brick(128, 128, 128)
    yield cube, r
    r.close()


@pytest.mark.parametrize("pose_index,tf_name", [(0, "a"), (17, "a"), (45, "b"), (100, "a")])
def test_hi_orbit_pose_sampled(hi, pose_index, tf_name):
    import torch
    cube, r = hi
    tf = synth.tf_hi_a() if tf_name == "a" else synth.tf_hi_b()
    cam = synth.orbit((1024, 1024, 2048), 120, 15.0, 1920, 1080)[pose_index]
    r.set_transfer_function(tf)
    r.set_camera(cam)
    img = r.render().cpu().numpy().astype(np.float64).reshape(-1, 4)
    W, H = 1920, 1080
    rng = np.random.default_rng(pose_index)
    rand = rng.integers(0, W * H, 3000)
    jj, ii = np.meshgrid(np.arange(H // 2 - 24, H // 2 + 24), np.arange(W // 2 - 24, W // 2 + 24),
                         indexing="ij")
    crop = (jj * W + ii).reshape(-1)
    pix = np.concatenate([rand, crop])
    ref, amb, ns = oracle.render(cube, tf, cam, brick=(128, 128, 128), pixels=pix,
                                 amb_alpha=AMB_ALPHA, amb_steps=AMB_STEPS)
    assert ns.sum() > 1e6
    assert_parity(img[pix], ref, amb, min_signal=0.01)
    st = r.stats()
    assert st["device_errors"] == 0
