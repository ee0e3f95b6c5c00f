"""FP64 CPU oracle for the bricked volume ray caster -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product library shares no code with
it and never calls it.

``vr_oracle.c`` is the plain FP64 ray caster (camera, slab entry/exit, fixed
step sampling, tri-linear interpolation, piecewise-linear transfer function,
opacity correction, front-to-back compositing with early termination, bricked
mode with per-brick runs folded by 'over', and the two-level fold of per-region
runs for sort-last distribution over ranks; Sections 1.2, 2.3.2-2.3.4 of
Hassan, Fluke & Barnes, arXiv:1205.0282).  ``quant.py`` builds the cube that
FP16 / FP8 storage reads back.  ``brute.py`` is an independent
arbitrary-precision restatement used to pin it on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB = os.path.join(_HERE, "_vr_oracle.so")
_lock = threading.Lock()
_lib = None

AMB_STEPS = 1
AMB_TERM = 2


class OrcCamera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fovy_deg", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("step", ctypes.c_double), ("term_alpha", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ``vr_oracle.c`` into ``oracle/_vr_oracle.so`` (gcc, OpenMP, no FMA
    contraction so that x86 and Arm hosts give identical results)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.orc_render.argtypes = [P, I64, I64, I64, P, ctypes.c_int32,
                                       ctypes.POINTER(OrcCamera), I64, I64, I64, ctypes.c_int32,
                                       ctypes.c_int32, P, I64, P, P, P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int32]
            lib.orc_render.restype = ctypes.c_int
            lib.orc_render_regions.argtypes = [P, I64, I64, I64, P, ctypes.c_int32,
                                               ctypes.POINTER(OrcCamera), I64, I64, I64, P, I64,
                                               P, I64, P, P, P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int32]
            lib.orc_render_regions.restype = ctypes.c_int
            lib.orc_pixel_ray.argtypes = [ctypes.POINTER(OrcCamera), I64, I64, I64,
                                          ctypes.c_int32, ctypes.c_int32, P]
            lib.orc_pixel_ray.restype = ctypes.c_int
            lib.orc_pixel_bricks.argtypes = [ctypes.POINTER(OrcCamera), I64, I64, I64, I64, I64,
                                             I64, P, I64, P, I64]
            lib.orc_pixel_bricks.restype = ctypes.c_int
            lib.orc_brick_minmax.argtypes = [P, I64, I64, I64, I64, I64, I64, P]
            lib.orc_brick_minmax.restype = ctypes.c_int
            lib.orc_tf_alpha_max.argtypes = [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
            lib.orc_tf_alpha_max.restype = ctypes.c_double
            _lib = lib
    return _lib


def _cam(c: dict) -> OrcCamera:
    oc = OrcCamera()
    oc.eye[:] = c["eye"]
    oc.target[:] = c["target"]
    oc.up[:] = c["up"]
    oc.fovy_deg = c["fovy_deg"]
    oc.width = c["width"]
    oc.height = c["height"]
    oc.step = c["step"]
    oc.term_alpha = c["term_alpha"]
    return oc


def _nbricks(shape_xyz, brick):
    return tuple((n - 1 + b - 1) // b for n, b in zip(shape_xyz, brick))


def render(cube: np.ndarray, tf: np.ndarray, cam: dict, brick=None, mode: str = "ea",
           pixels=None, amb_alpha: float = 1e-5, amb_steps: float = 1e-4, threads: int = 0,
           regions=None, step_mode: int = 0):
    """Render with the FP64 oracle.

    cube: float32[nz][ny][nx].  brick: (bx, by, bz) or None for monolithic.
    pixels: None for the whole image, else an int array of j*W+i indices.
    regions: None, or the region of every brick (brick id = ix + nbx*(iy + nby*iz);
    -1 = not rendered) for the two-level sort-last fold (needs a bricking and
    emission-absorption mode).
    step_mode: 0 fixed step; 1 dynamic step (samples cam["step"] voxels apart along
    each ray's dominant axis; not with regions).
    Returns (rgba, ambiguous_flags, samples): rgba is float64 (H, W, 4) for the
    whole image or (npix, 4) for a pixel list, premultiplied.
    """
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    nz, ny, nx = cube.shape
    tfa = np.ascontiguousarray(tf, dtype=np.float64).reshape(-1, 5)
    W, H = cam["width"], cam["height"]
    if pixels is None:
        npix = W * H
        pix_ptr = None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = len(pixels)
        pix_ptr = pixels.ctypes.data
    out = np.zeros((npix, 4), dtype=np.float64)
    amb = np.zeros(npix, dtype=np.uint8)
    samples = np.zeros(npix, dtype=np.int64)
    bx, by, bz = brick if brick is not None else (0, 0, 0)
    m = {"ea": 0, "mip": 1}[mode]
    oc = _cam(cam)
    if regions is not None:
        if brick is None or mode != "ea" or step_mode:
            raise ValueError("regions need a bricking and emission-absorption mode")
        reg = np.ascontiguousarray(regions, dtype=np.int32).reshape(-1)
        rc = _load().orc_render_regions(cube.ctypes.data, nx, ny, nz, tfa.ctypes.data, len(tfa),
                                        ctypes.byref(oc), bx, by, bz, reg.ctypes.data, len(reg),
                                        pix_ptr, npix, out.ctypes.data, amb.ctypes.data,
                                        samples.ctypes.data, amb_alpha, amb_steps, threads)
    else:
        rc = _load().orc_render(cube.ctypes.data, nx, ny, nz, tfa.ctypes.data, len(tfa),
                                ctypes.byref(oc), bx, by, bz, m, int(step_mode), pix_ptr, npix, out.ctypes.data,
                                amb.ctypes.data, samples.ctypes.data, amb_alpha, amb_steps, threads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    if pixels is None:
        return out.reshape(H, W, 4), amb.reshape(H, W), samples.reshape(H, W)
    return out, amb, samples


def pixel_ray(cam: dict, shape_xyz, i: int, j: int) -> dict:
    """Direction, entry/exit parameters, entry point and sample count of one pixel."""
    out = np.zeros(9, dtype=np.float64)
    oc = _cam(cam)
    hit = _load().orc_pixel_ray(ctypes.byref(oc), *shape_xyz, i, j, out.ctypes.data)
    return {"hit": bool(hit), "d": out[0:3].copy(), "t0": out[3], "t1": out[4],
            "p_entry": out[5:8].copy(), "n": int(out[8])}


def pixel_bricks(cam: dict, shape_xyz, brick, pixels) -> np.ndarray:
    """Bool (npix, n_bricks): which bricks own at least one sample of each pixel."""
    nb = _nbricks(shape_xyz, brick)
    n_bricks = nb[0] * nb[1] * nb[2]
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    mask = np.zeros((len(pixels), n_bricks), dtype=np.uint8)
    oc = _cam(cam)
    rc = _load().orc_pixel_bricks(ctypes.byref(oc), *shape_xyz, *brick, pixels.ctypes.data,
                                  len(pixels), mask.ctypes.data, n_bricks)
    if rc != 0:
        raise ValueError("bad brick arguments")
    return mask.astype(bool)


def brick_minmax(cube: np.ndarray, brick) -> np.ndarray:
    """float32 (n_bricks, 2): [min, max] over each brick's voxels plus its apron."""
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    nz, ny, nx = cube.shape
    nb = _nbricks((nx, ny, nz), brick)
    out = np.zeros((nb[0] * nb[1] * nb[2], 2), dtype=np.float32)
    rc = _load().orc_brick_minmax(cube.ctypes.data, nx, ny, nz, *brick, out.ctypes.data)
    if rc != 0:
        raise ValueError("bad brick arguments")
    return out


def tf_alpha_max(tf: np.ndarray, lo: float, hi: float) -> float:
    tfa = np.ascontiguousarray(tf, dtype=np.float64).reshape(-1, 5)
    return _load().orc_tf_alpha_max(tfa.ctypes.data, len(tfa), lo, hi)
