"""CPU checks of the seeded generator's block source (synth.BlockSource), the
input of the brick-provider load: any block equals the same voxels of the whole
cube bit for bit, through the native provider entry point with padded row and
slice strides too, and the ~200 GiB cube's blocks are deterministic.  The
generator holds no rendering arithmetic; it only makes inputs."""
import ctypes

import numpy as np
import pytest

import synth

SHAPE = (45, 38, 51)
SEED = 23


@pytest.fixture(scope="module")
def whole():
    return synth.hi_cube(seed=SEED, shape_xyz=SHAPE, n_line=20, n_cont=3)


@pytest.fixture(scope="module")
def source():
    return synth.BlockSource(SHAPE, SEED, synth.hi_sources(SEED, SHAPE, 20, 3))


def test_blocks_equal_the_whole_cube(whole, source):
    rng = np.random.default_rng(1)
    for _ in range(25):
        o = [int(rng.integers(0, n)) for n in SHAPE]
        e = [int(rng.integers(1, n - oo + 1)) for n, oo in zip(SHAPE, o)]
        blk = source.block(o, e)
        ref = whole[o[2]:o[2] + e[2], o[1]:o[1] + e[1], o[0]:o[0] + e[0]]
        assert np.array_equal(blk.view(np.uint32), ref.view(np.uint32))


def test_native_provider_entry_point_with_strides(whole, source):
    """The provider signature: voxel (i, j, k) of the box at dst[k*slice + j*row + i];
    the padding between rows and slices is left as it was."""
    fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                          ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_int64)(source.fn)
    o, e = (7, 30, 12), (33, 8, 20)
    row, slc = 40, 40 * 11
    buf = np.full(slc * e[2], -7.0, np.float32)
    rc = fn(source.user, (ctypes.c_int64 * 3)(*o), (ctypes.c_int32 * 3)(*e), buf.ctypes.data, row, slc)
    assert rc == 0
    got = np.lib.stride_tricks.as_strided(buf, shape=e[::-1], strides=(slc * 4, row * 4, 4))
    assert np.array_equal(got, whole[12:32, 30:38, 7:40])
    pad = buf.reshape(e[2], 11, 40)
    assert np.all(pad[:, :, 33:] == -7.0) and np.all(pad[:, 8:, :] == -7.0)
    # boxes outside the cube and short strides are refused
    assert fn(source.user, (ctypes.c_int64 * 3)(40, 0, 0), (ctypes.c_int32 * 3)(6, 1, 1), buf.ctypes.data, 8,
              8) != 0
    assert fn(source.user, (ctypes.c_int64 * 3)(0, 0, 0), (ctypes.c_int32 * 3)(4, 2, 1), buf.ctypes.data, 3,
              8) != 0


def test_xl_cube_is_a_deterministic_block_source():
    """4096 x 4096 x 3200 voxels from 100,500 sources; a brick's block is the same
    on every call and holds noise plus sources (never generated whole)."""
    src = synth.xl_source()
    assert src.shape_xyz == (4096, 4096, 3200) and len(src.sources) == 100_500
    a = src.block((2048, 1024, 3072), (65, 65, 65))
    b = src.block((2048, 1024, 3072), (65, 65, 65))
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert abs(float(a.mean())) < 0.05 and 0.9 < float(a.std()) < 1.5
    edge = src.block((4095 - 64, 4095 - 64, 3199 - 64), (65, 65, 65))
    assert np.isfinite(edge).all()


def test_fill_planes_writes_the_planes(whole, source):
    """The parallel plane filler (slabs for training on cubes larger than the
    device) writes the same voxels as the whole cube."""
    buf = np.full((9, SHAPE[1], SHAPE[0]), np.nan, np.float32)
    source.fill_planes(buf.ctypes.data, 30, 38, threads=3)
    assert np.array_equal(buf, whole[30:39])
