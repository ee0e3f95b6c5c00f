"""Reduced-precision storage of the cube -- TEST INFRASTRUCTURE (oracle side).

The paper samples FP32 sub-cubes.  The reduced-precision storage forms are an
extension: the cube is stored as FP16, or as FP8 E4M3 codes with one scale per
brick, and every sample reads back a value of that storage; interpolation,
transfer function and compositing are unchanged.  The image of such a render is
therefore defined as the image of the cube of read-back values, which is what
``stored_cube`` builds (the FP64 ray caster in ``vr_oracle.c`` then renders it).

Formats, written from their published definitions:

* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits;
  numpy's float32 -> float16 cast rounds to nearest, ties to even.
* OCP 8-bit floating point E4M3: 1 sign bit, 4 exponent bits (bias 7), 3
  mantissa bits; exponent field 0 holds the subnormals m/8 * 2^-6; S.1111.111 is
  NaN and there is no infinity, so the largest finite magnitude is
  1.75 * 2^8 = 448.  Encoding rounds to nearest, ties to even, saturating to
  +-448 ("satfinite").

Per-brick scale: voxel g along an axis of n voxels with brick side B lies in brick
min(g // B, nb - 1), nb = ceil((n - 1) / B) (the same bricking as the renderer,
Section 2.3.1); brick b's scale is s_b = float32(max |v| over its voxels) / 448 in
float32 (1 for an all-zero brick); voxel v is stored as the code of float32(v /
s_b) and reads back as float32(decode(code) * s_b).

Parity pins (tests/test_oracle_pins.py): the E4M3 table against values fixed by
the format (1.0, 448, the smallest subnormal 2^-9, the normal/subnormal edge),
exhaustive round-trip of every finite code, rounding of exact midpoints to the
even code, saturation, and brute-force nearest-value search on random inputs.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def e4m3_values() -> np.ndarray:
    """Value of each of the 256 E4M3 codes (NaN for 0x7f and 0xff)."""
    out = np.empty(256, dtype=np.float64)
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 0xF, code & 0x7
        if e == 0xF and m == 0x7:
            v = np.nan
        elif e == 0:
            v = (m / 8.0) * 2.0 ** -6
        else:
            v = (1.0 + m / 8.0) * 2.0 ** (e - 7)
        out[code] = -v if s else v
    return out


_POS = e4m3_values()[:127]  # codes 0x00..0x7e: 0, subnormals, normals up to 448 (increasing)


def e4m3_encode(x) -> np.ndarray:
    """E4M3 codes (uint8) of float32 values x: nearest finite value, ties to the
    even code, |x| >= 448 saturated to 448."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    if np.isnan(x).any():
        raise ValueError("NaN has no saturating E4M3 encoding here")
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.searchsorted(_POS, a, side="left")  # _POS[hi - 1] < a <= _POS[hi]
    hi = np.clip(hi, 0, 126)
    lo = np.maximum(hi - 1, 0)
    dlo = a - _POS[lo]
    dhi = _POS[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    code = np.where(a == _POS[hi], hi, code).astype(np.uint8)
    sign = (np.signbit(x) & (code != 0)).astype(np.uint8) << 7
    return (code | sign).astype(np.uint8)


def e4m3_decode(codes) -> np.ndarray:
    return e4m3_values()[np.asarray(codes, dtype=np.int64)]


def bricks_along(n: int, b: int) -> int:
    return max(1, (n - 1 + b - 1) // b)


def owner_index(n: int, b: int) -> np.ndarray:
    """Brick index along one axis of each voxel 0..n-1."""
    return np.minimum(np.arange(n) // b, bricks_along(n, b) - 1)


def brick_scales(cube: np.ndarray, brick) -> np.ndarray:
    """float32 [nbz][nby][nbx] per-brick scales of a float32 cube [z][y][x]."""
    cube = np.asarray(cube, dtype=np.float32)
    nz, ny, nx = cube.shape
    bx, by, bz = brick
    nb = (bricks_along(nx, bx), bricks_along(ny, by), bricks_along(nz, bz))
    ox, oy, oz = owner_index(nx, bx), owner_index(ny, by), owner_index(nz, bz)
    absmax = np.zeros((nb[2], nb[1], nb[0]), dtype=np.float32)
    a = np.abs(cube)
    for k in range(nb[2]):
        for j in range(nb[1]):
            for i in range(nb[0]):
                blk = a[np.ix_(oz == k, oy == j, ox == i)]
                absmax[k, j, i] = blk.max() if blk.size else 0.0
    s = absmax / np.float32(E4M3_MAX)
    return np.where(absmax > 0, s, np.float32(1.0)).astype(np.float32)


def stored_cube(cube: np.ndarray, precision: str, brick=None) -> np.ndarray:
    """The cube of values read back from `precision` storage ("f32", "f16", "f8";
    "f8" needs the bricking)."""
    cube = np.asarray(cube, dtype=np.float32)
    if precision == "f32":
        return cube.copy()
    if precision == "f16":
        return cube.astype(np.float16).astype(np.float32)
    if precision != "f8":
        raise ValueError(precision)
    nz, ny, nx = cube.shape
    s = brick_scales(cube, brick)
    bx, by, bz = brick
    sv = s[np.ix_(owner_index(nz, bz), owner_index(ny, by), owner_index(nx, bx))]
    q = (cube / sv).astype(np.float32)
    dec = e4m3_decode(e4m3_encode(q)).astype(np.float32)
    return (dec * sv).astype(np.float32)
