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


@pytest.mark.parametrize("shape,brick,cam", CASES)
def test_planned_tiles_are_sound(vrmod, shape, brick, cam):
    """Every pixel whose ray has samples in a brick (the oracle's ownership) lies
    in a tile the planner emits for that brick: culling tiles outside the brick's
    silhouette never drops work."""
    tiles = vrmod.vr_plan_brick_tiles(cam, shape, brick)
    rects = vrmod.vr_plan_brick_rects(cam, shape, brick)
    W, H = cam["width"], cam["height"]
    pixels = np.arange(W * H)
    owns = oracle.pixel_bricks(cam, shape, brick, pixels)
    tile = (pixels // W // 8) * ((W + 7) // 8) + (pixels % W) // 8
    for b in range(owns.shape[1]):
        hit = owns[:, b]
        assert np.all(tiles[b, tile[hit]]), f"brick {b}: a pixel with samples in a dropped tile"
        # and the tiles lie within the brick's rendering rectangle
        x0, y0, x1, y1 = rects[b]
        ty, tx = np.divmod(np.flatnonzero(tiles[b]), (W + 7) // 8)
        assert np.all((tx >= x0 // 8) & (tx <= x1 // 8) & (ty >= y0 // 8) & (ty <= y1 // 8))


def test_planned_tiles_drop_what_the_silhouette_misses(vrmod):
    """On the HI workload's 1080p orbit the silhouette test drops about a fifth of
    the rectangles' tiles (their corners), and keeps every tile a ray of the
    brick passes through (checked by exact ray-box tests of every pixel)."""
    shape, brick = (1024, 1024, 2048), (128, 128, 128)
    cam = synth.orbit(shape, 120, 15.0, 1920, 1080)[17]
    tiles = vrmod.vr_plan_brick_tiles(cam, shape, brick)
    rects = vrmod.vr_plan_brick_rects(cam, shape, brick)
    valid = rects[:, 2] >= rects[:, 0]
    rect_tiles = ((rects[:, 2] // 8 - rects[:, 0] // 8 + 1) * (rects[:, 3] // 8 - rects[:, 1] // 8 + 1))[valid].sum()
    kept = tiles.sum()
    assert kept < 0.9 * rect_tiles
    # exact check on a sample of bricks: every pixel whose ray meets the box keeps its tile
    eye, tgt, up = (np.asarray(cam[k], np.float64) for k in ("eye", "target", "up"))
    f = (tgt - eye) / np.linalg.norm(tgt - eye)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    W, H = cam["width"], cam["height"]
    th = np.tan(np.radians(cam["fovy_deg"]) / 2)
    jj, ii = np.mgrid[0:H, 0:W]
    d = f + ((2 * (ii + 0.5) / W - 1) * th * W / H)[..., None] * r + ((1 - 2 * (jj + 0.5) / H) * th)[..., None] * u
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    tile = (jj // 8) * ((W + 7) // 8) + ii // 8
    nb = [(n - 2 + b) // b for n, b in zip(shape, brick)]
    for b in np.random.default_rng(0).choice(np.flatnonzero(valid), 24, replace=False):
        ix, iy, iz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
        lo = np.array([ix, iy, iz], np.float64) * 128
        hi = np.minimum(lo + 128, np.array(shape) - 1)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - eye) / d, (hi - eye) / d
        tn, tf = np.minimum(t1, t2).max(-1), np.maximum(t1, t2).min(-1)
        hit = tf > np.maximum(tn, 0.0)
        assert np.all(tiles[b, tile[hit]]), b


def test_rectangles_are_tight_enough(vrmod):
    """Rectangles are not the whole screen: the planner actually culls."""
    cam = synth.tiny_views(width=256, height=256)[0]
    rects = vrmod.vr_plan_brick_rects(cam, (64, 64, 64), (16, 16, 16))
    area = ((rects[:, 2] - rects[:, 0] + 1) * (rects[:, 3] - rects[:, 1] + 1)).mean()
    assert area < 0.1 * 256 * 256


# ------------------------------------------------ the camera as OpenGL matrices

def _look_at(eye, target, up):
    """gluLookAt's modelview matrix (row r, column c)."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = (target - eye) / np.linalg.norm(target - eye)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def _perspective(fovy_deg, aspect, near=1.0, far=1e5):
    """gluPerspective's projection matrix (row r, column c)."""
    g = 1.0 / np.tan(np.radians(fovy_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0], p[1, 1] = g / aspect, g
    p[2, 2], p[2, 3] = (far + near) / (near - far), 2.0 * far * near / (near - far)
    p[3, 2] = -1.0
    return p


@pytest.mark.parametrize("k", range(4))
def test_camera_from_opengl_matrices(vrmod, k):
    """The viewer's modelview and projection matrices give the camera they were
    built from: the same eye, viewing direction, up and field of view, so the
    same rays (the planner's rendering rectangles agree to the pixel)."""
    shape, brick = (61, 47, 53), (16, 16, 16)
    cam = synth.tiny_views(seed=7 + k, width=(160, 96, 200, 64)[k], height=(90, 96, 150, 120)[k])[0]
    cam = dict(cam, eye=tuple(np.asarray(cam["eye"]) * (0.9 + 0.1 * k)))
    view = _look_at(cam["eye"], cam["target"], cam["up"])
    proj = _perspective(cam["fovy_deg"], cam["width"] / cam["height"])
    got = vrmod.vr_camera_from_matrices(view, proj, cam["width"], cam["height"], cam["step"], cam["term_alpha"])
    np.testing.assert_allclose(got["eye"], cam["eye"], rtol=1e-12, atol=1e-9)
    f0 = np.subtract(cam["target"], cam["eye"])
    f1 = np.subtract(got["target"], got["eye"])
    np.testing.assert_allclose(f1 / np.linalg.norm(f1), f0 / np.linalg.norm(f0), atol=1e-12)
    assert abs(got["fovy_deg"] - cam["fovy_deg"]) < 1e-9
    assert np.dot(got["up"], f1) == pytest.approx(0.0, abs=1e-12)
    assert np.dot(got["up"], cam["up"]) > 0.0
    want = vrmod.vr_plan_brick_rects(cam, (61, 47, 53), brick)
    assert np.array_equal(vrmod.vr_plan_brick_rects(got, shape, brick), want)
    # the column-major form is accepted as 16 values too
    got16 = vrmod.vr_camera_from_matrices(view.T.reshape(16), proj.T.reshape(16), cam["width"], cam["height"])
    np.testing.assert_allclose(got16["eye"], got["eye"], rtol=0, atol=0)


def test_camera_matrices_are_checked(vrmod):
    view = _look_at((100.0, 40.0, -80.0), (30.0, 20.0, 25.0), (0.0, 1.0, 0.0))
    proj = _perspective(35.0, 4.0 / 3.0)
    vrmod.vr_camera_from_matrices(view, proj, 640, 480)
    bad = []
    v = view.copy()
    v[0, :3] *= 1.01                      # not a rotation
    bad.append((v, proj, 640, 480))
    p = proj.copy()
    p[0, 2] = 0.1                         # off-centre frustum
    bad.append((view, p, 640, 480))
    bad.append((view, proj, 640, 640))    # aspect differs from the image's
    p = proj.copy()
    p[3, 3] = 1.0                         # orthographic-like, not a perspective
    bad.append((view, p, 640, 480))
    v = view.copy()
    v[3, 0] = 0.5                         # not affine
    bad.append((v, proj, 640, 480))
    for v, p, w, h in bad:
        with pytest.raises(vrmod.VRError) as e:
            vrmod.vr_camera_from_matrices(v, p, w, h)
        assert e.value.code == vrmod.VR_EINVAL
