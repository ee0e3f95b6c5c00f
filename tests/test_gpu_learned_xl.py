"""GPU test of the learned form's large-cube flow (bench.py --config xl) on a
small instance of the same recipe: the 4096x4096x3200 cube divided by 16 per
axis (256x256x200, its sources divided by 16^3), generated brick by brick on
request, the codec trained slab by slab, and the learned and plain out-of-core
forms rendered from the provider at two device budgets.  The flow must finish,
report no device errors, and render the learned frames within the PSNR the
fallback bound gives against the plain ones; with every brick cached both forms
render the same bricks."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_learned_form_on_a_cube_generated_on_request():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--config", "xl", "--learned", "--tf", "b",
           "--xl-scale", "16", "--xl-budgets-gib", "0.002,1", "--xl-frames", "2", "--xl-slab-layers", "1",
           "--xl-decoder-slabs", "2", "--train-steps", "300", "--xl-slab-steps", "200",
           "--train-batch", "65536", "--width", "320", "--height", "180", "--codec-brick", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    final = lines[-1]
    budgets = final["xl"]["budgets"]
    assert [b["budget_gib"] for b in budgets] == [0.002, 1.0]
    small, large = budgets
    for row in budgets:
        for form in ("plain", "learned"):
            assert row[form]["device_errors"] == 0
            assert row[form]["fps"] > 0
        assert row["learned"]["bricks_rendered_per_frame"] == row["plain"]["bricks_rendered_per_frame"] > 0
        assert 0 < row["learned"]["bricks_plain"] < row["learned"]["bricks"]
        assert row["psnr_db_learned_vs_plain"] is None or row["psnr_db_learned_vs_plain"] > 40.0
    # a small cache refills bricks every frame; a large one keeps them
    assert small["plain"]["bricks_filled_per_frame"] > 0
    assert large["plain"]["bricks_filled_per_frame"] == 0 and large["learned"]["bricks_filled_per_frame"] == 0
    nbz = (200 - 2 + 32) // 32       # brick layers of 32 over 200 planes
    assert final["xl"]["train_s"] > 0 and len(final["xl"]["loss_latents_last_per_slab"]) == nbz
