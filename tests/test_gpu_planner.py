"""GPU parity of the per-frame planner on a grid large enough for its threaded
paths: 15,525 bricks of 8^3 (the brick loop in eight chunks, the key-order
scatter of every chunk) and over 131,072 (brick, tile) items per frame (items
written by rows of tiles on several host threads).  The in-core image matches
the FP64 oracle on sampled pixels; the out-of-core context renders it bit for
bit, with every brick cached and with a cache that streams most bricks through
its ring (items written straight into launch order), frame after frame."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import AMB_ALPHA, AMB_STEPS, assert_parity

pytestmark = pytest.mark.gpu

SHAPE = (200, 184, 216)
BRICK = (8, 8, 8)              # 25 x 23 x 27 = 15,525 bricks
W, H = 1280, 960


@pytest.fixture(scope="module")
def case():
    cube = synth.hi_cube(seed=5, shape_xyz=SHAPE, n_line=60, n_cont=4)
    tf = synth.tf_tiny()
    cams = [synth.pose(SHAPE, a, e, W, H) for a, e in ((0.5, 0.35), (2.8, -0.5), (4.4, 1.1))]
    return cube, tf, cams


def test_threaded_plan_matches_the_oracle_and_out_of_core(case):
    import torch
    from paper_1205_0282_gb300 import vr
    cube, tf, cams = case
    want = []
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_TEX)
        r.brick(*BRICK)
        r.set_transfer_function(tf)
        for cam in cams:
            r.set_camera(cam)
            r.reset_stats()
            want.append(r.render().cpu().numpy())
            st = r.stats()
            assert st["device_errors"] == 0
            assert st["items"] > 131072 and st["bricks_rendered"] > 8 * 256
    rng = np.random.default_rng(3)
    for cam, img in zip(cams[:2], want[:2]):
        pix = rng.integers(0, W * H, 400)
        ref, amb, ns = oracle.render(cube, tf, cam, brick=BRICK, pixels=pix, amb_alpha=AMB_ALPHA,
                                     amb_steps=AMB_STEPS)
        assert ns.sum() > 10000
        assert_parity(img.astype(np.float64).reshape(-1, 4)[pix], ref, amb)
    slot = (BRICK[0] + 1) * (BRICK[1] + 1) * (BRICK[2] + 1) * 4 * 4
    for budget_bricks in (0, 3000):
        with vr.VolumeRenderer(0) as r:
            r.load_cube_host(cube)
            r.set_option(vr.VR_OPT_OOC_MARCH, 1)
            if budget_bricks:
                r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget_bricks * slot)
            r.brick(*BRICK)
            r.set_transfer_function(tf)
            for k in range(4):
                cam = cams[k % 3]
                r.set_camera(cam)
                r.reset_stats()
                got = r.render().cpu().numpy()
                st = r.stats()
                assert st["device_errors"] == 0
                assert np.array_equal(got, want[k % 3]), (budget_bricks, k)
                assert st["bricks_uploaded"] + st["bricks_cached"] == st["bricks_rendered"]
                if budget_bricks:
                    assert st["bricks_uploaded"] > st["bricks_rendered"] // 2   # streamed
                elif k == 3:
                    assert st["bricks_uploaded"] == 0
