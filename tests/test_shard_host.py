"""Host logic of the sort-last distribution, no GPU: the k-d partition of the
brick grid (Section 2.3.1), the visibility order of its leaves, and the
rendering rectangle of a leaf (Section 2.3.2), through the C ABI."""
import itertools

import numpy as np
import pytest

import synth
from paper_1205_0282_gb300 import vr

SHAPES = [((1024, 1024, 2048), (128, 128, 128)), ((64, 64, 64), (16, 16, 16)),
          ((61, 47, 53), (24, 16, 20)), ((300, 40, 90), (32, 8, 16))]


def _nb(shape, brick):
    return [(n - 1 + b - 1) // b for n, b in zip(shape, brick)]


@pytest.mark.parametrize("shape,brick", SHAPES)
@pytest.mark.parametrize("parts", [1, 2, 3, 4, 5, 6, 7, 8])
def test_partition_tiles_the_brick_grid(shape, brick, parts):
    nb = _nb(shape, brick)
    if parts > nb[0] * nb[1] * nb[2]:
        with pytest.raises(vr.VRError):
            vr.vr_kd_partition(shape, brick, parts)
        return
    R = vr.vr_kd_partition(shape, brick, parts)
    owner = -np.ones(nb[::-1], dtype=np.int64)   # [z][y][x]
    for k, (x0, y0, z0, x1, y1, z1) in enumerate(R):
        assert 0 <= x0 < x1 <= nb[0] and 0 <= y0 < y1 <= nb[1] and 0 <= z0 < z1 <= nb[2]
        box = owner[z0:z1, y0:y1, x0:x1]
        assert (box == -1).all(), "leaves overlap"
        box[...] = k
    assert (owner >= 0).all(), "leaves leave bricks uncovered"


def test_partition_is_balanced_and_cuts_the_longest_axis():
    # HI cube: 8 x 8 x 16 bricks; two parts cut z (longest) in half
    R = vr.vr_kd_partition((1024, 1024, 2048), (128, 128, 128), 2)
    assert R.tolist() == [[0, 0, 0, 8, 8, 8], [0, 0, 8, 8, 8, 16]]
    # eight parts: equal volumes
    R = vr.vr_kd_partition((1024, 1024, 2048), (128, 128, 128), 8)
    vols = [(r[3] - r[0]) * (r[4] - r[1]) * (r[5] - r[2]) for r in R]
    assert vols == [128] * 8
    # three parts: the low side takes one part and a third of the longest axis
    R = vr.vr_kd_partition((1024, 1024, 2048), (128, 128, 128), 3)
    assert R[0].tolist() == [0, 0, 0, 8, 8, 5]
    vols = sorted((r[3] - r[0]) * (r[4] - r[1]) * (r[5] - r[2]) for r in R)
    assert max(vols) / min(vols) < 1.25
    # ties between axes go to the lower axis
    R = vr.vr_kd_partition((65, 65, 65), (16, 16, 16), 2)
    assert R.tolist() == [[0, 0, 0, 2, 4, 4], [2, 0, 0, 4, 4, 4]]


def _leaves_of(R, B, P):
    """Leaf number of each point of P (n x 3, voxel coordinates), -1 if none."""
    out = -np.ones(len(P), dtype=np.int64)
    for k, r in enumerate(R):
        lo = np.array(r[:3]) * B
        hi = np.array(r[3:]) * B
        inside = ((P >= lo) & (P < hi)).all(axis=1)
        out[inside] = k
    return out


@pytest.mark.parametrize("shape,brick", SHAPES[1:])
@pytest.mark.parametrize("parts", [2, 3, 5, 8])
def test_order_is_front_to_back_along_every_ray(shape, brick, parts):
    """Walk random rays from random eyes (outside and inside the cube) in small
    steps: the leaves a ray meets must appear in the returned order."""
    rng = np.random.default_rng(parts)
    R = vr.vr_kd_partition(shape, brick, parts)
    nb = _nb(shape, brick)
    B = np.array(brick, dtype=np.float64)
    # brick-grid extent used by the leaves (the last brick may be shorter)
    hi = np.array([nb[a] * brick[a] for a in range(3)], dtype=np.float64)
    t = np.linspace(0.0, 3.0 * hi.max(), 3000)
    for _ in range(12):
        eye = rng.uniform(-0.5, 1.5, 3) * hi
        order = vr.vr_kd_order(shape, brick, parts, eye)
        assert sorted(order.tolist()) == list(range(parts))
        pos = np.empty(parts, dtype=np.int64)
        pos[order] = np.arange(parts)
        for _ in range(40):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            leaves = _leaves_of(R, B, eye[None, :] + t[:, None] * d[None, :])
            leaves = leaves[leaves >= 0]
            runs = leaves[np.r_[True, leaves[1:] != leaves[:-1]]] if len(leaves) else leaves
            ranks = pos[runs]
            assert (np.diff(ranks) > 0).all(), (eye, d, runs, order)   # in order, one run each


def test_region_rect_contains_its_bricks_rects():
    shape, brick = (61, 47, 53), (24, 16, 20)
    nb = _nb(shape, brick)
    R = vr.vr_kd_partition(shape, brick, 3)
    for cam in synth.tiny_views(width=90, height=70) + [synth.pose(shape, 1.0, 0.2, 90, 70)]:
        rects = vr.vr_plan_brick_rects(cam, shape, brick)
        for r in R:
            rr = vr.vr_plan_region_rect(cam, shape, brick, r[:3], r[3:])
            for x, y, z in itertools.product(range(r[0], r[3]), range(r[1], r[4]), range(r[2], r[5])):
                b = rects[x + nb[0] * (y + nb[1] * z)]
                if b[2] < b[0]:
                    continue
                assert rr[0] <= b[0] and rr[1] <= b[1] and rr[2] >= b[2] and rr[3] >= b[3]
        # the whole grid as one region is the union of all brick rectangles
        whole = vr.vr_plan_region_rect(cam, shape, brick, (0, 0, 0), nb)
        vis = rects[rects[:, 2] >= rects[:, 0]]
        assert whole.tolist() == [vis[:, 0].min(), vis[:, 1].min(), vis[:, 2].max(), vis[:, 3].max()]


def test_bad_arguments_are_rejected():
    with pytest.raises(vr.VRError):
        vr.vr_kd_partition((64, 64, 64), (16, 16, 16), 0)
    with pytest.raises(vr.VRError):
        vr.vr_kd_partition((64, 64, 64), (64, 64, 64), 2)   # one brick cannot be cut
    with pytest.raises(vr.VRError):
        vr.vr_plan_region_rect(synth.tiny_views()[0], (64, 64, 64), (16, 16, 16), (0, 0, 0), (5, 4, 4))
