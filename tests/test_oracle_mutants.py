"""The oracle's pins are strong enough to catch plausible slips.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), builds it, swaps it in for the real oracle library,
and runs the pin tests of test_oracle_pins.py against it: at least one pin
must fail.  The real oracle is untouched.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "vr_oracle.c")

MUTANTS = {
    "transposed x/z in trilinear": ("i0[2] * sz + i0[1] * sy + i0[0] * sx",
                                    "i0[0] * sz + i0[1] * sy + i0[2] * sx"),
    "dropped transmittance": ("double w = (1.0 - seg[3]) * alpha;", "double w = alpha;"),
    "inverted opacity-correction exponent": ("pow(1.0 - a, dt / 1.0)", "pow(1.0 - a, 1.0 / dt)"),
    "image rows bottom-up": ("(1.0 - 2.0 * (j + 0.5) / c->height)",
                             "(2.0 * (j + 0.5) / c->height - 1.0)"),
    "fold in back-to-front order": ("for (int ch = 0; ch < 4; ++ch) acc[ch] += t * seg[ch];",
                                    "double ts = 1.0 - seg[3]; (void)t; "
                                    "for (int ch = 0; ch < 4; ++ch) acc[ch] = seg[ch] + ts * acc[ch];"),
    "transfer-function weight reversed": ("double w = (v - p0[0]) / (p1[0] - p0[0]);",
                                          "double w = (p1[0] - v) / (p1[0] - p0[0]);"),
    "z weight flipped": ("return c0 + f[2] * (c1 - c0);", "return c1 + f[2] * (c0 - c1);"),
    "brick owner by ceil": ("int64_t b = (int64_t)floor(q / (double)J->brick[a]);",
                            "int64_t b = (int64_t)ceil(q / (double)J->brick[a]);"),
    "entry not clamped at the eye": ("double t0 = tn > 0.0 ? tn : 0.0, t1 = tf;",
                                     "double t0 = tn, t1 = tf;"),
    "closed sampling interval": ("if (!(s < L)) break;\n        double p[3];\n        for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];\n        int64_t b",
                                 "if (s > L) break;\n        double p[3];\n        for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];\n        int64_t b"),
    "aspect ratio dropped": ("* b->tan_half * b->aspect;", "* b->tan_half;"),
}


def _pin_calls():
    import json
    cases = json.load(open(pins.GOLDEN))["cases"]
    calls = [(f"hand:{c['name']}", lambda c=c: pins.test_hand_examples(c)) for c in cases]
    calls += [
        ("constant", lambda: pins.test_constant_cube_closed_form(0.5, 0.3, 0.99)),
        ("affine", pins.test_affine_field_closed_form),
        ("mip", pins.test_mip_affine_is_endpoint_max),
        ("opengl", pins.test_camera_matches_opengl_matrices),
        ("brute-mono", lambda: pins.test_brute_force_tiny(1, (4, 4, 4), None, 0.99, 0.6)),
        ("brute-brick", lambda: pins.test_brute_force_tiny(3, (4, 3, 4), (1, 2, 3), 0.99, 0.95)),
    ]
    return calls


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not found exactly once"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-o", str(so), str(mpath), "-lm"], check=True)
    real = oracle._load()
    mlib = ctypes.CDLL(str(so))
    for fn in ("orc_render", "orc_pixel_ray", "orc_pixel_bricks", "orc_brick_minmax",
               "orc_tf_alpha_max"):
        getattr(mlib, fn).argtypes = getattr(real, fn).argtypes
        getattr(mlib, fn).restype = getattr(real, fn).restype
    monkeypatch.setattr(oracle, "_lib", mlib)
    caught = []
    for pin_name, call in _pin_calls():
        try:
            call()
        except AssertionError:
            caught.append(pin_name)
    assert caught, f"no pin caught the planted mistake {name!r}"


def test_unmutated_copy_passes_all_pins(tmp_path, monkeypatch):
    """Control: the same harness with the unchanged source fails nothing."""
    so = tmp_path / "same.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-o", str(so), SRC, "-lm"], check=True)
    real = oracle._load()
    lib = ctypes.CDLL(str(so))
    for fn in ("orc_render", "orc_pixel_ray", "orc_pixel_bricks", "orc_brick_minmax",
               "orc_tf_alpha_max"):
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        getattr(lib, fn).restype = getattr(real, fn).restype
    monkeypatch.setattr(oracle, "_lib", lib)
    for _, call in _pin_calls():
        call()
