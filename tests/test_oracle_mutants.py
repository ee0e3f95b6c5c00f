"""The oracle's pins are strong enough to catch plausible slips.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), builds it, swaps it in for the real oracle library,
and runs the pin tests of test_oracle_pins.py against it: at least one pin
must fail.  The real oracle is untouched.  The pins run in a child process, so
that a mutant that reads out of bounds and crashes (which also counts as caught)
cannot take the test session down.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

if __name__ == "__main__":
    sys.path[:0] = [os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    os.path.dirname(os.path.abspath(__file__))]

import oracle  # noqa: E402
import test_oracle_pins as pins  # noqa: E402

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
    "region runs folded past termination": ("if (racc[3] < tau) fold(racc, seg);", "fold(racc, seg);"),
    "region run not restarted": ("racc[0] = racc[1] = racc[2] = racc[3] = 0.0;", "(void)racc;"),
    "dynamic step scaled the wrong way": ("dt = J->step_mode ? cam->step / dmax : cam->step",
                                          "dt = J->step_mode ? cam->step * dmax : cam->step"),
    "dynamic step from the entry": ("        t0 += 0.5 * dt;\n", "        t0 += 0.0 * dt;\n"),
    "region folded behind the pixel": ("if (acc[3] < tau) fold(acc, racc);\n                            near_tau",
                                       "if (acc[3] < tau) { double t_[4]; memcpy(t_, racc, sizeof(t_)); "
                                       "fold(t_, acc); memcpy(acc, t_, sizeof(t_)); }\n                            near_tau"),
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
        ("region-single", pins.test_region_fold_with_a_single_region_is_the_bricked_render),
        ("region-over", lambda: pins.test_region_fold_is_the_over_of_the_region_renders(2)),
        ("region-bound", pins.test_region_termination_bound),
        ("dynamic-axis", pins.test_dynamic_step_samples_the_middles_of_voxel_slabs),
        ("dynamic-closed", lambda: pins.test_dynamic_step_closed_form_on_a_constant_cube(1.0)),
    ]
    return calls


def _swap_in(so_path):
    """Load the library at so_path with the real oracle's signatures and make the
    oracle package use it."""
    real = oracle._load()
    lib = ctypes.CDLL(str(so_path))
    for fn in ("orc_render", "orc_render_regions", "orc_pixel_ray", "orc_pixel_bricks",
               "orc_brick_minmax", "orc_tf_alpha_max"):
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        getattr(lib, fn).restype = getattr(real, fn).restype
    oracle._lib = lib


def _run_pins_in_child(so_path):
    """(return code, names of the pins that failed) for the library at so_path."""
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(so_path)], cwd=here,
                       capture_output=True, text=True, timeout=600)
    caught = []
    for line in r.stdout.splitlines():
        if line.startswith("CAUGHT "):
            caught = json.loads(line[len("CAUGHT "):])
    return r.returncode, caught


def _build(src_text, tmp_path, name):
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src_text)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-o", str(so), str(cpath), "-lm"], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not found exactly once"
    so = _build(src.replace(old, new), tmp_path, "mutant")
    rc, caught = _run_pins_in_child(so)
    assert rc != 0 or caught, f"no pin caught the planted mistake {name!r}"


def test_unmutated_copy_passes_all_pins(tmp_path):
    """Control: the same harness with the unchanged source fails nothing."""
    so = _build(open(SRC).read(), tmp_path, "same")
    rc, caught = _run_pins_in_child(so)
    assert rc == 0 and caught == []


if __name__ == "__main__":
    # child: run every pin against the library given on the command line
    _swap_in(sys.argv[1])
    failed = []
    for pin_name, call in _pin_calls():
        try:
            call()
        except AssertionError:
            failed.append(pin_name)
    print("CAUGHT " + json.dumps(failed), flush=True)
