"""Pins for the FP64 oracle: it is checked against things other than itself.

* hand-derived worked examples (tests/golden/hand_examples.json);
* closed forms: a constant cube (A = 1-(1-alpha)^n, C = c*A, with and without
  termination) and an affine field (tri-linear interpolation reproduces it
  exactly, so the composited sum is an arithmetico-geometric series);
* the camera against the textbook OpenGL lookAt/perspective matrices that the
  paper's viewer passes (Section 2.3.2);
* brute force at 50 digits (oracle/brute.py) on 2^3..4^3 cubes, monolithic
  and bricked, with termination active;
* invariants: bricked == monolithic with termination off; with it on, the
  bricked result is never below and at most 1 - term_alpha above (the
  compositing operator is associative, Section 2.3.3); a 90 degree rotation
  of cube and camera together; per-brick min/max against numpy.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _cube5(kind):
    if kind == "constant 2.0":
        return np.full((5, 5, 5), 2.0, dtype=np.float32)
    if kind == "value = z":
        z = np.arange(5, dtype=np.float32)
        return np.broadcast_to(z[:, None, None], (5, 5, 5)).copy()
    raise KeyError(kind)


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_examples(case):
    cam = synth.camera((2, 2, -10), (2, 2, 2), (0, 1, 0), 30.0, 1, 1, step=case["step"],
                       term_alpha=case["term_alpha"])
    brick = tuple(case["brick"]) if case["brick"] else None
    rgba, amb, ns = oracle.render(_cube5(case["cube"]), np.array(case["tf"]), cam, brick=brick,
                                  mode=case["mode"])
    np.testing.assert_allclose(rgba[0, 0], case["expected"], rtol=0, atol=1e-15)
    # the same worked example through the independent brute force
    if case["mode"] == "ea":
        b, _ = brute.render(_cube5(case["cube"]), np.array(case["tf"]), cam, brick=brick)
        np.testing.assert_allclose(b[0], case["expected"], rtol=0, atol=1e-15)


# ------------------------------------------------------------------ closed forms

def _alpha(a, dt):
    return 1.0 - (1.0 - a) ** dt


@pytest.mark.parametrize("dt,a,tau", [(0.5, 0.02, 1.0), (0.5, 0.3, 0.99), (1.0, 0.1, 0.99),
                                      (0.25, 0.6, 0.95), (0.7, 0.05, 0.99)])
def test_constant_cube_closed_form(dt, a, tau):
    """V = v0 everywhere: every composited sample has the same alpha, so a ray
    with n samples gives A = 1 - (1-alpha)^n_eff, C = c*A, where n_eff is n
    cut at the first k with 1-(1-alpha)^k >= tau."""
    v0 = 1.5
    cube = np.full((20, 24, 28), v0, dtype=np.float32)   # nz, ny, nx
    col = np.array([0.9, 0.4, 0.2])
    tf = np.array([[0.0, *col, a], [3.0, *col, a]])
    cam = synth.pose((28, 24, 20), 0.6, 0.3, 48, 40, step=dt, term_alpha=tau)
    rgba, amb, ns = oracle.render(cube, tf, cam)
    al = _alpha(a, dt)
    n_term = math.ceil(math.log(1.0 - tau) / math.log(1.0 - al)) if tau < 1.0 else 10 ** 9
    hit = ns > 0
    assert hit.sum() > 500
    # the per-pixel sample count the oracle reports is the geometric count, capped
    for j in range(0, 40, 7):
        for i in range(0, 48, 5):
            r = oracle.pixel_ray(cam, (28, 24, 20), i, j)
            assert ns[j, i] == min(r["n"], n_term)
    A = 1.0 - (1.0 - al) ** ns
    np.testing.assert_allclose(rgba[..., 3], A, rtol=0, atol=1e-13)
    for c in range(3):
        np.testing.assert_allclose(rgba[..., c], col[c] * A, rtol=0, atol=1e-13)


def test_axis_ray_sample_count():
    """A ray along +z through voxel centres, entering at z = 0: n = ceil((nz-1)/dt)."""
    for nz, dt in [(5, 0.5), (17, 0.5), (16, 0.3), (9, 1.0), (33, 0.7)]:
        cam = synth.camera((2, 2, -10), (2, 2, 2), (0, 1, 0), 30.0, 1, 1, step=dt)
        r = oracle.pixel_ray(cam, (5, 5, nz), 0, 0)
        np.testing.assert_allclose(r["d"], [0, 0, 1], atol=0)
        assert r["t0"] == 10.0 and r["t1"] == 10.0 + nz - 1
        assert r["n"] == math.ceil((nz - 1) / dt - 1e-12)


def _series(q, n, r0, r1):
    """sum_{k<n} q^k (r0 + k r1), summed directly in fp64 long hand."""
    k = np.arange(n, dtype=np.float64)
    return float(np.sum(q ** k * (r0 + k * r1)))


def test_affine_field_closed_form():
    """V = gx*x + gy*y + gz*z + e is reproduced exactly by tri-linear
    interpolation, so sample k has value v(p_entry) + k dt (g.d).  With a
    constant opacity and a colour linear in v, the composited red channel is
    alpha * sum_k (1-alpha)^k r(v_k), an arithmetico-geometric series.  The
    gradient differs per axis, so a transposed axis or a wrong sample position
    breaks it."""
    nx, ny, nz = 23, 19, 17
    gx, gy, gz, e = 0.25, -0.5, 0.125, 1.0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = (gx * x + gy * y + gz * z + e).astype(np.float32)
    lo, hi = -20.0, 20.0
    a0 = 0.03
    tf = np.array([[lo, 0.0, 1.0, 0.5, a0], [hi, 1.0, 0.0, 0.5, a0]])
    dt = 0.5
    cam = synth.pose((nx, ny, nz), 2.1, -0.35, 40, 36, step=dt, term_alpha=1.0)
    rgba, amb, ns = oracle.render(cube, tf, cam)
    al = _alpha(a0, dt)
    g = np.array([gx, gy, gz])
    checked = 0
    for j in range(0, 36, 3):
        for i in range(0, 40, 3):
            r = oracle.pixel_ray(cam, (nx, ny, nz), i, j)
            n = r["n"]
            if n == 0:
                assert np.all(rgba[j, i] == 0)
                continue
            v0 = float(g @ r["p_entry"] + e)
            dv = dt * float(g @ r["d"])
            r0 = (v0 - lo) / (hi - lo)
            r1 = dv / (hi - lo)
            red = al * _series(1.0 - al, n, r0, r1)
            green = al * _series(1.0 - al, n, 1.0 - r0, -r1)
            A = 1.0 - (1.0 - al) ** n
            np.testing.assert_allclose(rgba[j, i], [red, green, 0.5 * A, A], rtol=0, atol=1e-12)
            checked += 1
    assert checked > 60


def test_mip_affine_is_endpoint_max():
    """Along a ray an affine field is monotone, so its maximum over the samples
    is at the first or the last sample (maximum intensity projection, the
    paper's own transfer function, Section 2.3.3)."""
    nx, ny, nz = 21, 18, 15
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cube = (0.5 * x - 0.25 * y + 0.375 * z).astype(np.float32)
    tf = np.array([[-10.0, 0.0, 0.2, 1.0, 0.0], [20.0, 1.0, 0.6, 0.0, 1.0]])
    cam = synth.pose((nx, ny, nz), 0.9, 0.5, 32, 32, step=0.5)
    rgba, amb, ns = oracle.render(cube, tf, cam, mode="mip")
    g = np.array([0.5, -0.25, 0.375])
    for j in range(0, 32, 4):
        for i in range(0, 32, 4):
            r = oracle.pixel_ray(cam, (nx, ny, nz), i, j)
            if r["n"] == 0:
                assert np.all(rgba[j, i] == 0)
                continue
            v_first = g @ r["p_entry"]
            v_last = g @ (r["p_entry"] + (r["n"] - 1) * 0.5 * r["d"])
            vm = max(v_first, v_last)
            w = (vm + 10.0) / 30.0
            exp = np.array([w, 0.2 + 0.4 * w, 1.0 - w, w])
            exp[:3] *= exp[3]
            np.testing.assert_allclose(rgba[j, i], exp, rtol=0, atol=1e-12)


# ------------------------------------------------------------- camera vs OpenGL

def _look_at(eye, centre, up):
    f = np.asarray(centre, float) - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    M = np.eye(4)
    M[0, :3], M[1, :3], M[2, :3] = s, u, -f
    M[:3, 3] = -M[:3, :3] @ eye
    return M


def _perspective(fovy_deg, aspect, near, far):
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    return np.array([[f / aspect, 0, 0, 0], [0, f, 0, 0],
                     [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)],
                     [0, 0, -1, 0]])


def test_camera_matches_opengl_matrices():
    """The paper's viewer sends OpenGL projection and model-view matrices
    (Section 2.3.2).  Each oracle pixel ray, pushed through the textbook
    lookAt/perspective matrices, must land on that pixel's centre in NDC
    (row 0 at the top of the image)."""
    shape = (30, 20, 40)
    for az, el, W, H in [(0.3, 0.2, 64, 48), (2.5, -0.7, 33, 57), (4.0, 1.1, 80, 20)]:
        cam = synth.pose(shape, az, el, W, H, fovy_deg=37.0)
        eye = np.array(cam["eye"])
        MVP = _perspective(37.0, W / H, 1.0, 1e4) @ _look_at(eye, cam["target"], cam["up"])
        for j in range(0, H, 5):
            for i in range(0, W, 7):
                r = oracle.pixel_ray(cam, shape, i, j)
                P = np.append(eye + 100.0 * r["d"], 1.0)
                clip = MVP @ P
                ndc = clip[:2] / clip[3]
                np.testing.assert_allclose(ndc, [2 * (i + .5) / W - 1, 1 - 2 * (j + .5) / H],
                                           atol=1e-12)


def test_entry_exit_on_box_faces():
    """Entry and exit points lie on the domain's surface (or the entry is the
    eye when it is inside); the sample count is #{k : k dt < t1 - t0}."""
    shape = (31, 17, 25)
    ext = np.array(shape, float) - 1
    cams = [synth.pose(shape, 1.0, 0.4, 24, 24),
            synth.camera((15, 8, 12), (30, 2, 1), (0, 1, 0), 60.0, 24, 24)]  # eye inside
    for cam in cams:
        eye = np.array(cam["eye"])
        inside = np.all((eye >= 0) & (eye <= ext))
        for j in range(24):
            for i in range(24):
                r = oracle.pixel_ray(cam, shape, i, j)
                if not r["hit"]:
                    continue
                pin = r["p_entry"]
                pout = eye + r["t1"] * r["d"]
                for p, may_be_eye in ((pin, inside), (pout, False)):
                    assert np.all(p >= -1e-9) and np.all(p <= ext + 1e-9)
                    on_face = np.any(np.isclose(p, 0, atol=1e-9) | np.isclose(p, ext, atol=1e-9))
                    assert on_face or (may_be_eye and np.allclose(p, eye))
                L = r["t1"] - r["t0"]
                assert r["n"] == int(np.sum(np.arange(r["n"] + 2) * cam["step"] < L))


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("seed,shape,brick,tau,amax", [
    (1, (4, 4, 4), None, 0.99, 0.6),
    (2, (4, 4, 4), (2, 2, 2), 0.99, 0.6),
    (3, (4, 3, 4), (1, 2, 3), 0.99, 0.95),
    (4, (3, 3, 3), None, 0.9, 0.95),
    (5, (2, 2, 2), (1, 1, 1), 0.99, 0.99),
    (6, (4, 4, 2), (3, 1, 1), 1.0, 0.5),
])
def test_brute_force_tiny(seed, shape, brick, tau, amax):
    cube = synth.random_cube(shape, seed)
    tf = synth.make_tf([0.0, 0.6 * amax, 0.95 * amax, amax], lo=-1.0, hi=5.0)
    rng = np.random.default_rng(seed)
    cams = [synth.pose(shape, rng.uniform(0, 6.3), rng.uniform(-1.2, 1.2), 9, 7, fovy_deg=40.0,
                       step=0.5, term_alpha=tau),
            # eye inside the box
            synth.camera((np.array(shape) - 1) * 0.3, (np.array(shape) - 1) * 0.9, (0, 1, 0), 80.0,
                         7, 6, step=0.35, term_alpha=tau)]
    peak = 0.0
    for cam in cams:
        a, amb, ns = oracle.render(cube, tf, cam, brick=brick)
        b, fl = brute.render(cube, tf, cam, brick=brick)
        a = a.reshape(-1, 4)
        ok = (amb.reshape(-1) == 0) & (fl == 0)
        assert ok.sum() >= 0.8 * len(ok)
        np.testing.assert_allclose(a[ok], b[ok], rtol=0, atol=1e-12)
        peak = max(peak, a[:, 3].max())
    assert peak > 0.3


def test_termination_really_triggers_in_brute_cases():
    """Guard: the brute-force cases exercise early termination (some rays stop
    before their last sample)."""
    cube = synth.random_cube((4, 4, 4), 2)
    tf = synth.make_tf([0.0, 0.6 * 0.95, 0.95 * 0.95, 0.95], lo=-1.0, hi=5.0)
    cam = synth.pose((4, 4, 4), 1.0, 0.3, 9, 7, fovy_deg=40.0, step=0.5)
    rgba, amb, ns = oracle.render(cube, tf, cam)
    geo = np.array([[oracle.pixel_ray(cam, (4, 4, 4), i, j)["n"] for i in range(9)]
                    for j in range(7)])
    assert np.any((ns < geo) & (ns > 0))


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("brick", [(1, 1, 1), (2, 2, 2), (4, 4, 4), (8, 8, 8), (16, 16, 16),
                                   (24, 24, 24), (32, 16, 8)])
def test_bricking_invariant(brick):
    """Termination off: any bricking composited with 'over' equals the
    monolithic render (associativity, Section 2.3.3).  Termination at 0.99:
    bricked >= monolithic and the excess is at most 1 - 0.99."""
    cube = synth.tiny_cube()
    tf = synth.tf_tiny()
    for tau in (1.0, 0.99):
        for cam in synth.tiny_views(width=48, height=40, term_alpha=tau)[:2]:
            mono, amb_m, _ = oracle.render(cube, tf, cam)
            brk, amb_b, _ = oracle.render(cube, tf, cam, brick=brick)
            if tau == 1.0:
                np.testing.assert_allclose(brk, mono, rtol=0, atol=1e-12)
            else:
                diff = brk - mono
                assert diff.min() >= -1e-12
                assert diff.max() <= 1.0 - tau + 1e-12


def test_bricking_invariant_is_not_vacuous():
    """With an opaque transfer function the per-brick termination does change
    the result (so the inequality above is exercised, not trivially equal)."""
    cube = synth.tiny_cube()
    tf = synth.make_tf([0.0, 0.0, 0.3, 0.6, 0.8, 0.9, 0.95, 0.99])
    cam = synth.tiny_views(width=48, height=40)[0]
    mono, _, _ = oracle.render(cube, tf, cam)
    brk, _, _ = oracle.render(cube, tf, cam, brick=(8, 8, 8))
    d = brk - mono
    assert d.max() > 1e-4 and d.min() >= -1e-12 and d.max() <= 0.01 + 1e-12


def test_rotation_invariance():
    """Rotating the cube by 90 degrees about y together with the camera gives
    the same image."""
    cube = synth.tiny_cube()[:, :, :48]             # nz=64, ny=64, nx=48 (not cubic)
    nz, ny, nx = cube.shape
    tf = synth.tf_tiny()
    cam = synth.pose((nx, ny, nz), 0.8, 0.3, 40, 30)
    # new cube R[z', y, x'] with x' = z, z' = nx-1-x : a rotation about +y
    rot = np.ascontiguousarray(np.transpose(cube, (2, 1, 0))[::-1])
    def rotp(p):
        return (p[2], p[1], (nx - 1) - p[0])
    cam_r = dict(cam)
    cam_r["eye"] = rotp(cam["eye"])
    cam_r["target"] = rotp(cam["target"])
    cam_r["up"] = (0.0, 1.0, 0.0)
    a, amb_a, _ = oracle.render(cube, tf, cam)
    b, amb_b, _ = oracle.render(rot, tf, cam_r)
    ok = (amb_a == 0) & (amb_b == 0)
    np.testing.assert_allclose(a[ok], b[ok], rtol=0, atol=1e-9)
    assert np.abs(a).max() > 0.1


def test_zero_opacity_and_missing_rays():
    cube = synth.tiny_cube()
    tf = synth.tf_tiny().copy()
    tf[:, 4] = 0.0
    cam = synth.tiny_views(width=32, height=32)[1]
    rgba, _, _ = oracle.render(cube, tf, cam)
    assert np.all(rgba == 0.0)
    away = synth.camera((31.5, 31.5, -100.0), (31.5, 31.5, -200.0), (0, 1, 0), 30.0, 16, 16)
    rgba, _, ns = oracle.render(cube, synth.tf_tiny(), away)
    assert np.all(rgba == 0.0) and np.all(ns == 0)


def test_single_voxel_spike_symmetric():
    """A spike at the centre of a zero cube, viewed head-on along z through its
    centre with an even image, gives an image symmetric under x and y flips."""
    n = 9
    cube = np.zeros((n, n, n), dtype=np.float32)
    cube[4, 4, 4] = 8.0
    tf = np.array([[0.0, 0.0, 0.0, 0.0, 0.0], [8.0, 1.0, 0.5, 0.25, 0.8]])
    cam = synth.camera((4, 4, -20), (4, 4, 4), (0, 1, 0), 20.0, 20, 20)
    rgba, _, _ = oracle.render(cube, tf, cam)
    assert rgba[..., 3].max() > 0.05
    np.testing.assert_allclose(rgba, rgba[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(rgba, rgba[::-1, :], atol=1e-13)


def test_brick_minmax_matches_numpy():
    cube = synth.tiny_cube()
    for brick in [(32, 32, 32), (24, 16, 40), (7, 9, 11)]:
        mm = oracle.brick_minmax(cube, brick)
        nb = [(64 - 1 + b - 1) // b for b in brick]
        k = 0
        for iz in range(nb[2]):
            for iy in range(nb[1]):
                for ix in range(nb[0]):
                    sl = cube[iz * brick[2]: min((iz + 1) * brick[2], 63) + 1,
                              iy * brick[1]: min((iy + 1) * brick[1], 63) + 1,
                              ix * brick[0]: min((ix + 1) * brick[0], 63) + 1]
                    assert mm[k, 0] == sl.min() and mm[k, 1] == sl.max()
                    k += 1


def test_tf_alpha_max_matches_dense_sampling():
    tf = synth.tf_hi_b()
    rng = np.random.default_rng(0)
    for _ in range(50):
        lo, hi = np.sort(rng.uniform(-5, 12, 2))
        grid = np.concatenate([np.linspace(lo, hi, 20001), tf[:, 0][(tf[:, 0] > lo) & (tf[:, 0] < hi)]])
        dense = np.interp(grid, tf[:, 0], tf[:, 4]).max()
        assert abs(oracle.tf_alpha_max(tf, lo, hi) - dense) < 1e-12
    assert oracle.tf_alpha_max(tf, -3.0, 6.5) == 0.0
    assert oracle.tf_alpha_max(tf, -3.0, 6.6) > 0.0


# ------------------------------------------------------------ storage quantisers
from oracle import quant  # noqa: E402


def test_e4m3_table_fixed_points():
    """Values the E4M3 definition fixes (1 sign, 4 exponent bits with bias 7, 3
    mantissa bits, subnormals at exponent field 0, S.1111.111 = NaN)."""
    v = quant.e4m3_values()
    assert v[0x38] == 1.0 and v[0xB8] == -1.0
    assert v[0x7E] == 448.0 and v[0xFE] == -448.0
    assert v[0x01] == 2.0 ** -9 and v[0x07] == 7 * 2.0 ** -9
    assert v[0x08] == 2.0 ** -6 and v[0x3F] == 1.875 and v[0x40] == 2.0
    assert v[0x00] == 0.0 and np.signbit(v[0x80])
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    assert np.isnan(v).sum() == 2
    pos = v[:127]
    assert np.all(np.diff(pos) > 0)  # codes 0..0x7e increase
    assert np.allclose(v[128:255], -v[:127])


def test_e4m3_round_trip_and_ties():
    v = quant.e4m3_values()
    finite = [c for c in range(256) if not np.isnan(v[c]) and c != 0x80]
    assert list(quant.e4m3_encode(v[finite])) == finite
    # exact midpoints go to the even code
    assert quant.e4m3_encode(1.0625) == 0x38   # between 1.0 (0x38) and 1.125 (0x39)
    assert quant.e4m3_encode(1.1875) == 0x3A   # between 1.125 (0x39) and 1.25 (0x3a)
    assert quant.e4m3_encode(2.0 ** -10) == 0x00   # between 0 and 2^-9
    assert quant.e4m3_encode(3 * 2.0 ** -10) == 0x02
    assert quant.e4m3_encode(15 * 2.0 ** -10) == 0x08   # subnormal 7/8 2^-6 | normal 2^-6
    assert quant.e4m3_encode(np.nextafter(np.float32(1.0625), np.float32(2))) == 0x39
    # saturation
    assert quant.e4m3_encode(464.0) == 0x7E and quant.e4m3_encode(1e30) == 0x7E
    assert quant.e4m3_encode(-1e6) == 0xFE


def test_e4m3_encode_is_the_nearest_value_brute_force():
    rng = np.random.default_rng(5)
    x = (rng.choice([-1, 1], 4000) * 2.0 ** rng.uniform(-12, 9.5, 4000)).astype(np.float32)
    codes = quant.e4m3_encode(x)
    v = quant.e4m3_values()
    fin = np.array([c for c in range(256) if not np.isnan(v[c])])
    for xi, c in zip(x.astype(np.float64), codes):
        xs = np.clip(xi, -448, 448)
        d = np.abs(v[fin] - xs)
        best = fin[d == d.min()]
        best_vals = set(v[best])
        assert v[c] in best_vals or (v[c] == 0 and 0.0 in best_vals)
        if len(best_vals) > 1:  # a tie: the even mantissa wins
            assert c % 2 == 0


def test_fp16_storage_fixed_points():
    c = np.array([[[1 / 3, 65504.0, 2.0 ** -24, 1.0 + 2.0 ** -11]]], dtype=np.float32)
    s = quant.stored_cube(c, "f16")
    assert s[0, 0, 0] == np.float32(0.333251953125)
    assert s[0, 0, 1] == 65504.0 and s[0, 0, 2] == 2.0 ** -24
    assert s[0, 0, 3] == 1.0  # tie between 1 and 1 + 2^-10 goes to the even fraction


def test_brick_ownership():
    assert list(quant.owner_index(9, 4)) == [0, 0, 0, 0, 1, 1, 1, 1, 1]
    assert list(quant.owner_index(10, 4)) == [0, 0, 0, 0, 1, 1, 1, 1, 2, 2]
    assert list(quant.owner_index(5, 8)) == [0] * 5


def fp8_lossless_cube(shape_xyz, brick, seed=7):
    """A cube that FP8 storage holds exactly: per brick b a power-of-two scale 2^k_b,
    every value a finite E4M3 value times 2^k_b, and one voxel of magnitude
    448 * 2^k_b so that the brick's scale is exactly 2^k_b."""
    nx, ny, nz = shape_xyz
    cube = synth.hi_cube(seed=seed, shape_xyz=shape_xyz, n_line=12, n_cont=2)
    ox, oy, oz = (quant.owner_index(n, b) for n, b in zip(shape_xyz, brick))
    kb = -5 - ((ox[None, None, :] + oy[None, :, None] + oz[:, None, None]) % 3)
    scale = np.ldexp(np.float32(1), kb).astype(np.float32)
    q = quant.e4m3_decode(quant.e4m3_encode(cube / scale)).astype(np.float32) * scale
    for k in range(oz.max() + 1):
        for j in range(oy.max() + 1):
            for i in range(ox.max() + 1):
                z0, y0, x0 = np.argmax(oz == k), np.argmax(oy == j), np.argmax(ox == i)
                q[z0, y0, x0] = 448.0 * scale[z0, y0, x0]
    return q.astype(np.float32)


def test_fp8_storage_of_a_representable_cube_is_exact():
    for shape, brick in [((40, 33, 27), (16, 16, 8)), ((64, 64, 64), (32, 32, 32))]:
        c = fp8_lossless_cube(shape, brick)
        s = quant.brick_scales(c, brick)
        assert np.all(np.log2(s) == np.round(np.log2(s)))
        assert np.array_equal(quant.stored_cube(c, "f8", brick), c)


def test_fp8_storage_error_bound():
    """|read-back - v| <= 2^-4 |v| (3 mantissa bits, round to nearest) plus half
    the subnormal spacing 2^-10 s_b, and each brick keeps its largest magnitude."""
    c = synth.tiny_cube()
    brick = (24, 20, 32)
    q = quant.stored_cube(c, "f8", brick)
    s = quant.brick_scales(c, brick)
    nz, ny, nx = c.shape
    sv = s[np.ix_(quant.owner_index(nz, brick[2]), quant.owner_index(ny, brick[1]),
                  quant.owner_index(nx, brick[0]))]
    err = np.abs(q.astype(np.float64) - c)
    assert np.all(err <= 2.0 ** -4 * np.abs(c) + 2.0 ** -10 * sv + 1e-6 * np.abs(c))
    assert err.max() > 0
    # relative error of the normal range is well inside the bound on average
    assert np.median(err / np.maximum(np.abs(c), 1e-30)) < 2.0 ** -5


# ------------------------------------------------------- two-level (region) fold

def _region_map(nb, split_axis, split_at):
    """Two regions of a brick grid nb (x, y, z), split at brick index split_at."""
    ids = np.arange(nb[0] * nb[1] * nb[2])
    idx = np.stack([ids % nb[0], (ids // nb[0]) % nb[1], ids // (nb[0] * nb[1])], axis=1)
    return (idx[:, split_axis] >= split_at).astype(np.int32)


def _over(images):
    """Front-to-back 'over' fold of RGBA images (no termination)."""
    acc = np.zeros_like(images[0])
    for im in images:
        acc = acc + (1.0 - acc[..., 3:4]) * im
    return acc


@pytest.mark.parametrize("tau", [1.0, 0.99])
def test_region_fold_with_one_region_per_brick_is_the_bricked_render(tau):
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)
    nb = [(64 - 1 + 16 - 1) // 16] * 3
    for cam in synth.tiny_views(width=40, height=36, term_alpha=tau)[:2]:
        ref, amb_r, _ = oracle.render(cube, tf, cam, brick=brick)
        got, amb_g, _ = oracle.render(cube, tf, cam, brick=brick,
                                      regions=np.arange(nb[0] * nb[1] * nb[2], dtype=np.int32))
        assert np.array_equal(got, ref) and np.array_equal(amb_g, amb_r)


def test_region_fold_with_a_single_region_is_the_bricked_render():
    cube = synth.tiny_cube()
    tf = synth.make_tf([0.0, 0.0, 0.3, 0.6, 0.8, 0.9, 0.95, 0.99])   # opaque: termination active
    brick = (8, 8, 8)
    cam = synth.tiny_views(width=40, height=36)[0]
    ref, _, _ = oracle.render(cube, tf, cam, brick=brick)
    got, _, _ = oracle.render(cube, tf, cam, brick=brick, regions=np.zeros(8 ** 3, dtype=np.int32))
    assert np.array_equal(got, ref)


def _three_regions(nb, axis):
    """Three slabs of a brick grid nb (x, y, z) along axis: bricks [0,1), [1,3), [3,...)."""
    ids = np.arange(nb[0] * nb[1] * nb[2])
    idx = np.stack([ids % nb[0], (ids // nb[0]) % nb[1], ids // (nb[0] * nb[1])], axis=1)[:, axis]
    return np.where(idx < 1, 0, np.where(idx < 3, 1, 2)).astype(np.int32)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_region_fold_is_the_over_of_the_region_renders(axis):
    """Termination off: rendering each of three slab regions alone (other bricks
    excluded) and folding the images front to back equals the full render
    (associativity, Section 2.3.3); the eye lies on the low side, so the low slab
    is in front."""
    cube, tf = synth.tiny_cube(), synth.tf_tiny()
    brick = (16, 16, 16)
    reg = _three_regions((4, 4, 4), axis)
    eye = [31.5, 31.5, 31.5]
    eye[axis] = -60.0
    target = [31.5, 31.5, 31.5]
    up = (0.0, 1.0, 0.0) if axis != 1 else (0.0, 0.0, 1.0)
    cam = synth.camera(eye, target, up, 40.0, 40, 36, term_alpha=1.0)
    full, _, _ = oracle.render(cube, tf, cam, brick=brick)
    three, _, _ = oracle.render(cube, tf, cam, brick=brick, regions=reg)
    parts = [oracle.render(cube, tf, cam, brick=brick, regions=np.where(reg == k, 0, -1))[0] for k in range(3)]
    np.testing.assert_allclose(three, full, rtol=0, atol=1e-12)
    np.testing.assert_allclose(_over(parts), full, rtol=0, atol=1e-12)
    assert np.abs(_over(parts[::-1]) - full).max() > 1e-3   # the order matters
    assert min(p[..., 3].max() for p in parts) > 0.02   # every slab contributes


def test_region_termination_bound():
    """Termination at tau < 1: each region stops on its own, so the two-level
    result differs from the bricked one by at most 1 - tau per channel, and the
    difference is not vacuous for an opaque transfer function."""
    cube = synth.tiny_cube()
    tf = synth.make_tf([0.0, 0.0, 0.3, 0.6, 0.8, 0.9, 0.95, 0.99])
    brick = (8, 8, 8)
    reg = _region_map((8, 8, 8), 2, 3)
    worst = 0.0
    for cam in synth.tiny_views(width=40, height=36)[:3]:
        ref, _, _ = oracle.render(cube, tf, cam, brick=brick)
        got, _, _ = oracle.render(cube, tf, cam, brick=brick, regions=reg)
        d = np.abs(got - ref)
        assert d.max() <= 1.0 - cam["term_alpha"] + 1e-12
        worst = max(worst, d.max())
    assert worst > 1e-4


# ------------------------------------------------------------------ dynamic step

def test_dynamic_step_samples_the_middles_of_voxel_slabs():
    """An axis-aligned ray (the centre pixel of an odd-sized image looking along
    +z) through the affine field v = z: with step 1 the dynamic samples sit at
    z = 0.5, 1.5, ..., n - 1.5 (the middles of the voxel slabs), the fixed ones at
    z = 0, 1, ..., n - 2; MIP returns the last sample's value."""
    n = 20
    z = np.arange(n, dtype=np.float32)
    cube = np.ascontiguousarray(np.broadcast_to(z[:, None, None], (n, n, n)))
    tf = np.array([[0.0, 1.0, 1.0, 1.0, 0.5], [40.0, 1.0, 1.0, 1.0, 0.5]])   # colour map of the MIP value
    cam = synth.camera((9.3, 8.7, -30.0), (9.3, 8.7, 10.0), (0, 1, 0), 20.0, 9, 7, step=1.0, term_alpha=1.0)
    pix = np.array([3 * 9 + 4])
    _, _, nd = oracle.render(cube, tf, cam, pixels=pix, step_mode=1)
    _, _, nf = oracle.render(cube, tf, cam, pixels=pix)
    assert nd[0] == n - 1 and nf[0] == n - 1
    lo = np.array([[0.0, 0.0, 0.0, 0.0, 0.0], [40.0, 1.0, 0.0, 0.0, 1.0]])   # red = opacity = value / 40
    md, _, _ = oracle.render(cube, lo, cam, pixels=pix, mode="mip", step_mode=1)
    mf, _, _ = oracle.render(cube, lo, cam, pixels=pix, mode="mip")
    # premultiplied: red = (v / 40) * (v / 40)
    assert abs(md[0, 0] - ((n - 1.5) / 40.0) ** 2) < 1e-12
    assert abs(mf[0, 0] - ((n - 2.0) / 40.0) ** 2) < 1e-12


@pytest.mark.parametrize("step", [0.5, 1.0])
def test_dynamic_step_closed_form_on_a_constant_cube(step):
    """Constant cube, termination off: after n samples spaced dt = step / max|d_a|
    from half a step after the entry the opacity is 1 - (1 - a)^(n dt), n = the
    count of (k + 1/2) dt < L (Section 2.3.2's discrete ray casting: one sample
    per `step` voxels along the dominant axis)."""
    cube = np.full((20, 20, 20), 2.0, dtype=np.float32)
    a_tf = 0.07
    tf = np.array([[0.0, 0.2, 0.4, 0.6, a_tf], [4.0, 0.2, 0.4, 0.6, a_tf]])
    cam = synth.camera((-15.0, 33.0, -9.0), (9.5, 9.5, 9.5), (0, 1, 0), 40.0, 17, 13, step=step,
                       term_alpha=1.0)
    rgba, _, ns = oracle.render(cube, tf, cam, step_mode=1)
    checked = 0
    for j in range(13):
        for i in range(17):
            ray = oracle.pixel_ray(cam, (20, 20, 20), i, j)
            if ray["n"] == 0:
                continue
            d = np.array(ray["d"])
            L = ray["t1"] - ray["t0"]
            dt = step / np.abs(d).max()
            n = 0
            while (n + 0.5) * dt < L:    # samples at (k + 1/2) dt < L
                n += 1
            assert ns[j, i] == n
            A = 1.0 - (1.0 - a_tf) ** (n * dt)
            assert abs(rgba[j, i, 3] - A) < 1e-12
            assert abs(rgba[j, i, 0] - 0.2 * A) < 1e-12
            checked += 1
    assert checked > 50
    # a diagonal view really takes fewer samples than the fixed step would
    _, _, nf = oracle.render(cube, tf, cam)
    assert ns.sum() < nf.sum()
