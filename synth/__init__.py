"""Seeded synthetic inputs shared by the GPU renderer's tests/bench and the oracle.

This module only *describes and generates inputs*: data cubes, transfer-function
control points and camera poses.  It holds none of the rendering method's
arithmetic, so both sides (the CUDA library and the FP64 oracle) can take their
inputs from it without sharing any part of the computation.

Workloads (stand-ins for the paper's survey cubes of Table 1, which are not
available; the axes follow an HI spectral cube, Section 1.1):

* ``tiny``: 64^3 cube = N(0,1) noise + 8 Gaussian sources (amplitude 3-10 sigma,
  spatial FWHM 2-6 voxels, spectral FWHM 2-12 voxels, uniform centres), 32^3
  bricks, 256x256 images at 4 seeded view angles, step 0.5 voxel, 8-point
  transfer function over [-3, 10] sigma, termination at alpha >= 0.99.
* ``hi``: 1024x1024x2048 cube (8 GiB) = noise + 2000 line sources (amplitude
  log-uniform 1-20 sigma, spectral FWHM 3-40 channels, spatial FWHM 2-6) + 50
  continuum sources extended along the whole spectral axis, 128^3 bricks,
  1920x1080 images, step 0.5, 16-point transfer functions, a 120-pose orbit
  about the y axis (the paper rotates its cubes about Y, Section 3.1).
* ``xl``: 4096x4096x3200 cube (~200 GiB) = noise + 100,000 line sources + 500
  continuum sources (the HI recipe), generated block by block on demand
  (``BlockSource``), never whole.

A camera is a plain dict with keys ``eye, target, up`` (3-tuples of float),
``fovy_deg``, ``width``, ``height``, ``step``, ``term_alpha``.  A transfer
function is a float64 array of shape (n, 5): rows ``(v, r, g, b, a)`` with v
strictly increasing, colours in [0, 1] and ``a`` the opacity per unit voxel of
path.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_gen.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None

FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def build(force: bool = False) -> str:
    """Compile the generator into ``synth/_synth.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O3", "-fno-math-errno", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_noise.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_uint64, ctypes.c_double]
            lib.synth_noise.restype = None
            lib.synth_add_sources.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
            lib.synth_add_sources.restype = None
            lib.synth_block.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
            lib.synth_block.restype = None
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------- cubes

def noise_cube(nx: int, ny: int, nz: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """float32[nz][ny][nx] of independent N(0, sigma^2) values (counter-based)."""
    cube = np.empty((nz, ny, nx), dtype=np.float32)
    _load().synth_noise(cube.ctypes.data, nx, ny, nz, seed, sigma)
    return cube


def add_sources(cube: np.ndarray, sources: np.ndarray) -> np.ndarray:
    """Add Gaussian sources in place; ``sources`` rows are
    (amplitude, x0, y0, z0, sigma_spatial, sigma_spectral, continuum_flag)."""
    assert cube.dtype == np.float32 and cube.flags.c_contiguous and cube.ndim == 3
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 7)
    nz, ny, nx = cube.shape
    if len(src):
        _load().synth_add_sources(cube.ctypes.data, nx, ny, nz, src.ctypes.data, len(src))
    return cube


def line_sources(rng: np.random.Generator, n: int, shape_xyz, amp, fwhm_sp, fwhm_sf,
                 log_amp: bool = False) -> np.ndarray:
    """Draw n line (3D Gaussian) sources with uniform random centres."""
    nx, ny, nz = shape_xyz
    if log_amp:
        a = np.exp(rng.uniform(math.log(amp[0]), math.log(amp[1]), n))
    else:
        a = rng.uniform(amp[0], amp[1], n)
    x0 = rng.uniform(0, nx, n)
    y0 = rng.uniform(0, ny, n)
    z0 = rng.uniform(0, nz, n)
    ss = rng.uniform(fwhm_sp[0], fwhm_sp[1], n) * FWHM_TO_SIGMA
    sf = rng.uniform(fwhm_sf[0], fwhm_sf[1], n) * FWHM_TO_SIGMA
    return np.stack([a, x0, y0, z0, ss, sf, np.zeros(n)], axis=1)


def continuum_sources(rng: np.random.Generator, n: int, shape_xyz, amp, fwhm_sp) -> np.ndarray:
    nx, ny, nz = shape_xyz
    a = np.exp(rng.uniform(math.log(amp[0]), math.log(amp[1]), n))
    x0 = rng.uniform(0, nx, n)
    y0 = rng.uniform(0, ny, n)
    ss = rng.uniform(fwhm_sp[0], fwhm_sp[1], n) * FWHM_TO_SIGMA
    return np.stack([a, x0, y0, np.zeros(n), ss, np.ones(n), np.ones(n)], axis=1)


def tiny_cube(seed: int = 1) -> np.ndarray:
    """64^3 noise + 8 Gaussian sources (amplitude 3-10, FWHM 2-6 / 2-12)."""
    n = 64
    cube = noise_cube(n, n, n, seed)
    rng = np.random.default_rng(seed)
    src = line_sources(rng, 8, (n, n, n), (3.0, 10.0), (2.0, 6.0), (2.0, 12.0))
    return add_sources(cube, src)


def hi_sources(seed: int = 3, shape_xyz=(1024, 1024, 2048), n_line: int = 2000,
               n_cont: int = 50) -> np.ndarray:
    """The source list of an HI-survey-like cube: line sources (amplitude
    log-uniform 1-20 sigma, spatial FWHM 2-6, spectral FWHM 3-40 channels), then
    continuum sources (amplitude log-uniform 1-20 sigma, spatial FWHM 2-6)."""
    rng = np.random.default_rng(seed)
    lines = line_sources(rng, n_line, shape_xyz, (1.0, 20.0), (2.0, 6.0), (3.0, 40.0),
                         log_amp=True)
    cont = continuum_sources(rng, n_cont, shape_xyz, (1.0, 20.0), (2.0, 6.0))
    return np.concatenate([lines, cont], axis=0)


def hi_cube(seed: int = 3, shape_xyz=(1024, 1024, 2048), n_line: int = 2000,
            n_cont: int = 50) -> np.ndarray:
    """HI-survey-like cube: noise + line sources + continuum sources.

    The full size (1024x1024x2048, 8 GiB) is the default; smaller shapes with
    proportionally fewer sources serve tests."""
    nx, ny, nz = shape_xyz
    cube = noise_cube(nx, ny, nz, seed)
    return add_sources(cube, hi_sources(seed, shape_xyz, n_line, n_cont))


def cube_block(shape_xyz, seed: int, sources: np.ndarray, origin, extent,
               sigma: float = 1.0) -> np.ndarray:
    """float32[ez][ey][ex] block at ``origin`` of the cube noise_cube(*shape_xyz,
    seed, sigma) + add_sources(sources), generated without the rest of the cube
    (bit for bit the same values)."""
    nx, ny, nz = shape_xyz
    o = np.ascontiguousarray(origin, dtype=np.int64)
    e = np.ascontiguousarray(extent, dtype=np.int32)
    assert all(o >= 0) and all(e >= 1) and all(o + e <= np.array(shape_xyz))
    src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 7)
    out = np.empty((int(e[2]), int(e[1]), int(e[0])), dtype=np.float32)
    _load().synth_block(out.ctypes.data, int(e[0]), int(e[0]) * int(e[1]), o.ctypes.data, e.ctypes.data,
                        nx, ny, nz, seed, sigma, src.ctypes.data, len(src))
    return out


class _CubeDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("seed", ctypes.c_uint64), ("sigma", ctypes.c_double),
                ("src", ctypes.c_void_p), ("n_src", ctypes.c_int64)]


class BlockSource:
    """A procedural cube as a native block source: ``fn`` is the address of a C
    function with the renderer library's brick-provider signature (origin,
    extent, destination, row and slice strides) and ``user`` the address of its
    cube description; both stay valid while this object lives.  Any thread may
    call it; nothing is held in memory but the source list."""

    def __init__(self, shape_xyz, seed: int, sources: np.ndarray, sigma: float = 1.0):
        lib = _load()
        self.shape_xyz = tuple(int(v) for v in shape_xyz)
        self.seed = int(seed)
        self.sources = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 7)
        self._desc = _CubeDesc((ctypes.c_int64 * 3)(*self.shape_xyz), self.seed, float(sigma),
                               self.sources.ctypes.data, len(self.sources))
        self.fn = ctypes.cast(lib.synth_cube_block, ctypes.c_void_p).value
        self.user = ctypes.addressof(self._desc)
        self._lib = lib

    def block(self, origin, extent) -> np.ndarray:
        return cube_block(self.shape_xyz, self.seed, self.sources, origin, extent, self._desc.sigma)

    def fill_planes(self, dst_ptr: int, z0: int, z1: int, threads: int = 0) -> None:
        """Write the planes z0..z1 (inclusive) of the cube, float32[z1-z0+1][ny][nx],
        to host memory at dst_ptr, split over threads (0: one per CPU)."""
        from concurrent.futures import ThreadPoolExecutor
        nx, ny, _ = self.shape_xyz
        fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_int64)(self.fn)
        plane = nx * ny
        # tasks of a quarter plane (rows), so that a thin slab still spreads over the threads
        rows = max(1, ny // 4)
        tasks = [(z, y) for z in range(z0, z1 + 1) for y in range(0, ny, rows)]

        def one(t):
            z, y = t
            h = min(rows, ny - y)
            o = (ctypes.c_int64 * 3)(0, y, z)
            e = (ctypes.c_int32 * 3)(nx, h, 1)
            rc = fn(self.user, o, e, dst_ptr + 4 * ((z - z0) * plane + y * nx), nx, plane)
            if rc:
                raise RuntimeError(f"block source failed ({rc})")

        with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
            list(ex.map(one, tasks))


def random_cube(shape_xyz, seed: int, lo: float = -2.0, hi: float = 6.0) -> np.ndarray:
    """Small cube of independent uniform values (for brute-force cases)."""
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (nz, ny, nx)).astype(np.float32)


# ------------------------------------------------------------------ transfer functions

def _ramp_colour(t: np.ndarray) -> np.ndarray:
    """Blue -> white -> red colour ramp over t in [0, 1]."""
    t = np.asarray(t, dtype=np.float64)
    r = np.where(t < 0.5, 2.0 * t, 1.0)
    g = np.where(t < 0.5, 2.0 * t, 2.0 - 2.0 * t)
    b = np.where(t < 0.5, 1.0, 2.0 - 2.0 * t)
    return np.stack([r, g, b], axis=1)


def make_tf(alpha, lo: float = -3.0, hi: float = 10.0) -> np.ndarray:
    """Uniformly spaced control points over [lo, hi] with the given opacities."""
    a = np.asarray(alpha, dtype=np.float64)
    n = len(a)
    v = lo + (hi - lo) * np.arange(n) / (n - 1)
    rgb = _ramp_colour(np.arange(n) / (n - 1))
    return np.concatenate([v[:, None], rgb, a[:, None]], axis=1)


def tf_tiny() -> np.ndarray:
    """8 points on [-3, 10] sigma; opacity zero up to 0.71 sigma."""
    return make_tf([0, 0, 0, 0.02, 0.05, 0.1, 0.2, 0.4])


def tf_hi_a() -> np.ndarray:
    """16 points on [-3, 10] sigma; opacity > 0 from about 0.5 sigma (noise visible)."""
    return make_tf([0, 0, 0, 0, 0, 0.005, 0.01, 0.02, 0.04, 0.06, 0.09, 0.13, 0.18, 0.24,
                    0.32, 0.4])


def tf_hi_b() -> np.ndarray:
    """16 points on [-3, 10] sigma; opacity zero below 6.5 sigma (empty-space skipping)."""
    return make_tf([0] * 12 + [0.1, 0.2, 0.3, 0.4])


# ---------------------------------------------------------------------------- cameras

def camera(eye, target, up=(0.0, 1.0, 0.0), fovy_deg=30.0, width=256, height=256,
           step=0.5, term_alpha=0.99) -> dict:
    return {"eye": tuple(float(x) for x in eye), "target": tuple(float(x) for x in target),
            "up": tuple(float(x) for x in up), "fovy_deg": float(fovy_deg),
            "width": int(width), "height": int(height), "step": float(step),
            "term_alpha": float(term_alpha)}


def framing(shape_xyz, fovy_deg=30.0):
    """Centre of the box [0, n-1]^3 and an eye distance that fits its bounding
    sphere inside the vertical field of view with 5% margin."""
    ext = np.array([s - 1 for s in shape_xyz], dtype=np.float64)
    centre = 0.5 * ext
    radius = 0.5 * float(np.linalg.norm(ext))
    dist = radius / math.sin(math.radians(fovy_deg / 2.0)) * 1.05
    return centre, dist


def pose(shape_xyz, azimuth, elevation, width, height, fovy_deg=30.0, **kw) -> dict:
    centre, dist = framing(shape_xyz, fovy_deg)
    d = np.array([math.cos(elevation) * math.sin(azimuth), math.sin(elevation),
                  math.cos(elevation) * math.cos(azimuth)])
    return camera(centre + dist * d, centre, (0.0, 1.0, 0.0), fovy_deg, width, height, **kw)


def tiny_views(seed: int = 2, n: int = 4, width: int = 256, height: int = 256, **kw):
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 2.0 * math.pi, n)
    el = rng.uniform(math.radians(-60.0), math.radians(60.0), n)
    return [pose((64, 64, 64), a, e, width, height, **kw) for a, e in zip(az, el)]


def orbit(shape_xyz, n_poses=120, elevation_deg=15.0, width=1920, height=1080, **kw):
    """n_poses camera poses evenly spaced in azimuth about the y axis."""
    el = math.radians(elevation_deg)
    return [pose(shape_xyz, 2.0 * math.pi * i / n_poses, el, width, height, **kw)
            for i in range(n_poses)]


# ----------------------------------------------------------------------- configurations

TINY = {"name": "tiny", "shape_xyz": (64, 64, 64), "brick": (32, 32, 32),
        "width": 256, "height": 256}
MID = {"name": "mid", "shape_xyz": (512, 512, 1024), "brick": (128, 128, 128),
       "width": 1920, "height": 1080}
HI = {"name": "hi", "shape_xyz": (1024, 1024, 2048), "brick": (128, 128, 128),
      "width": 1920, "height": 1080}
# ~200 GiB: never held whole in host memory; blocks come from BlockSource(XL ...)
XL = {"name": "xl", "shape_xyz": (4096, 4096, 3200), "brick": (128, 128, 128),
      "width": 1920, "height": 1080, "n_line": 100_000, "n_cont": 500, "seed": 7}


def xl_source() -> "BlockSource":
    """The 4096x4096x3200 cube (noise + 100k line + 500 continuum sources) as a
    block source."""
    return BlockSource(XL["shape_xyz"], XL["seed"],
                       hi_sources(XL["seed"], XL["shape_xyz"], XL["n_line"], XL["n_cont"]))
