"""Python binding of the C ABI in ``include/vr.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all rendering
work runs in ``libvr.so``'s CUDA kernels.  PyTorch is used only to hand over
device buffers and streams.  There is no fallback: if ``libvr.so`` is missing
the import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvr.so")

VR_OK = 0
VR_EINVAL = -1
VR_ENOMEM = -2
VR_ECUDA = -3
VR_ESTATE = -4
VR_ETIMEOUT = -5
VR_ESOURCE = -6

VR_OPT_SKIP_EMPTY = 1
VR_OPT_RECT_CULL = 2
VR_OPT_MODE = 3
VR_OPT_KERNEL = 4
VR_KERNEL_TMA = 0
VR_KERNEL_DIRECT = 1
VR_KERNEL_TEX = 2
VR_KERNEL_AUTO = 3
VR_OPT_PRECISION = 5
VR_OPT_DEVICE_BUDGET = 6
VR_OPT_STEP_MODE = 7
VR_OPT_TEX_SLAB_LAYERS = 8
VR_OPT_OOC_MARCH = 9
VR_OPT_PROVIDER_THREADS = 10
VR_OPT_HOST_OUTPUT_ASYNC = 11
VR_PRECISION_F32 = 0
VR_PRECISION_F16 = 1
VR_PRECISION_F8 = 2

_ERR_NAMES = {VR_EINVAL: "VR_EINVAL", VR_ENOMEM: "VR_ENOMEM", VR_ECUDA: "VR_ECUDA",
              VR_ESTATE: "VR_ESTATE", VR_ETIMEOUT: "VR_ETIMEOUT", VR_ESOURCE: "VR_ESOURCE"}


class VRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class vr_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fovy_deg", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("step", ctypes.c_double), ("term_alpha", ctypes.c_double)]


class vr_stats(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("items", ctypes.c_int64), ("fragments", ctypes.c_int64),
                ("bricks_rendered", ctypes.c_int64), ("bricks_skipped", ctypes.c_int64),
                ("touched_bytes", ctypes.c_int64), ("march_ms", ctypes.c_double),
                ("composite_ms", ctypes.c_double), ("frame_ms", ctypes.c_double),
                ("plan_ms", ctypes.c_double), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("chunks_staged", ctypes.c_int64), ("chunks_direct", ctypes.c_int64),
                ("bricks_uploaded", ctypes.c_int64), ("bricks_cached", ctypes.c_int64),
                ("device_errors", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# The exported symbols, in header order (tests check them against include/vr.h).
EXPORTS = ["vr_create", "vr_destroy", "vr_load_cube", "vr_load_cube_host", "vr_load_cube_provider", "vr_brick", "vr_set_transfer_function",
           "vr_set_camera", "vr_camera_from_matrices", "vr_set_camera_matrices", "vr_set_option", "vr_render", "vr_get_stats", "vr_reset_stats",
           "vr_get_brick_minmax", "vr_plan_brick_rects", "vr_plan_brick_tiles", "vr_kd_partition", "vr_kd_order",
           "vr_set_region", "vr_region_rect", "vr_plan_region_rect", "vr_render_rect",
           "vr_composite_subimages", "vr_server_create", "vr_server_submit", "vr_server_wait",
           "vr_server_get_stats", "vr_server_destroy", "vr_codec_gemm_check", "vr_codec_create",
           "vr_codec_destroy", "vr_codec_param_count", "vr_codec_set_params", "vr_codec_get_params",
           "vr_codec_forward", "vr_codec_gradient", "vr_codec_fit_stats", "vr_codec_train", "vr_codec_fit_stats_slab",
           "vr_codec_train_slab",
           "vr_codec_decode_bricks", "vr_codec_get_minmax", "vr_codec_brick_count", "vr_codec_brick_size",
           "vr_load_cube_codec", "vr_set_codec_fallback", "vr_set_codec_fallback_provider", "vr_codec_brick_errors", "vr_render_noalloc",
           "vr_last_error"]


class vr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_frames", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("items", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1205_0282_gb300.build` "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.vr_create.argtypes = [ctypes.POINTER(P), I32]
    lib.vr_destroy.argtypes = [P]
    lib.vr_destroy.restype = None
    lib.vr_server_destroy.restype = None
    lib.vr_codec_param_count.restype = ctypes.c_int64
    lib.vr_load_cube.argtypes = [P, P, I64, I64, I64]
    lib.vr_load_cube_host.argtypes = [P, P, I64, I64, I64]
    lib.vr_load_cube_provider.argtypes = [P, P, P, I64, I64, I64]
    lib.vr_brick.argtypes = [P, I32, I32, I32]
    lib.vr_set_transfer_function.argtypes = [P, P, I32]
    lib.vr_set_camera.argtypes = [P, ctypes.POINTER(vr_camera)]
    D = ctypes.c_double
    lib.vr_camera_from_matrices.argtypes = [P, P, I32, I32, D, D, ctypes.POINTER(vr_camera)]
    lib.vr_set_camera_matrices.argtypes = [P, P, P, I32, I32, D, D]
    lib.vr_set_option.argtypes = [P, I32, I64]
    lib.vr_render.argtypes = [P, P, P]
    lib.vr_get_stats.argtypes = [P, ctypes.POINTER(vr_stats)]
    lib.vr_reset_stats.argtypes = [P]
    lib.vr_get_brick_minmax.argtypes = [P, P, I64]
    lib.vr_plan_brick_rects.argtypes = [ctypes.POINTER(vr_camera), I64, I64, I64, I32, I32, I32,
                                        P, I64]
    lib.vr_plan_brick_tiles.argtypes = [ctypes.POINTER(vr_camera), I64, I64, I64, I32, I32, I32, P, I64, I64]
    lib.vr_kd_partition.argtypes = [I64, I64, I64, P, I32, P]
    lib.vr_kd_order.argtypes = [I64, I64, I64, P, I32, P, P]
    lib.vr_set_region.argtypes = [P, P, P]
    lib.vr_region_rect.argtypes = [P, P]
    lib.vr_plan_region_rect.argtypes = [ctypes.POINTER(vr_camera), I64, I64, I64, P, P, P, P]
    lib.vr_render_rect.argtypes = [P, P, P, P]
    lib.vr_composite_subimages.argtypes = [P, I32, P, P, P, P]
    lib.vr_server_create.argtypes = [P, I64, I32, ctypes.POINTER(P)]
    lib.vr_server_submit.argtypes = [P, ctypes.POINTER(vr_camera), P, I32, P, ctypes.POINTER(I64)]
    lib.vr_server_wait.argtypes = [P, I64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.vr_server_get_stats.argtypes = [P, ctypes.POINTER(vr_server_stats)]
    lib.vr_server_destroy.argtypes = [P]
    lib.vr_codec_gemm_check.argtypes = [P, P, I32, I32, I32, I32, P]
    lib.vr_codec_create.argtypes = [I32, P, ctypes.POINTER(P)]
    lib.vr_codec_destroy.argtypes = [P]
    lib.vr_codec_destroy.restype = None
    lib.vr_codec_param_count.argtypes = [P]
    lib.vr_codec_set_params.argtypes = [P, P, P, P]
    lib.vr_codec_get_params.argtypes = [P, P, P, P]
    lib.vr_codec_forward.argtypes = [P, P, I64, P]
    lib.vr_codec_gradient.argtypes = [P, P, P, I64, P, ctypes.POINTER(ctypes.c_double)]
    lib.vr_codec_fit_stats.argtypes = [P, P, I64, I64, I64, ctypes.c_float]
    lib.vr_codec_get_minmax.argtypes = [P, P]
    lib.vr_codec_brick_count.argtypes = [P]
    lib.vr_codec_brick_count.restype = I32
    lib.vr_codec_brick_size.argtypes = [P, P]
    lib.vr_codec_brick_size.restype = None
    lib.vr_load_cube_codec.argtypes = [P, P, I64, I64, I64]
    lib.vr_set_codec_fallback.argtypes = [P, P, ctypes.c_float, ctypes.c_float]
    lib.vr_set_codec_fallback_provider.argtypes = [P, P, P, ctypes.c_float, ctypes.c_float]
    lib.vr_codec_brick_errors.argtypes = [P, P, ctypes.POINTER(I64)]
    lib.vr_codec_train.argtypes = [P, P, I64, I64, I64, I32, I32, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_double)]
    lib.vr_codec_decode_bricks.argtypes = [P, P, P, I32, P, P]
    lib.vr_codec_fit_stats_slab.argtypes = [P, P, I64, I64, I64, I32, I32, ctypes.c_float]
    lib.vr_codec_train_slab.argtypes = [P, P, I64, I64, I64, I32, I32, I32, I32, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    lib.vr_render_noalloc.argtypes = [P, I64, I64, I64, I32, I32, I32, P, I32,
                                      ctypes.POINTER(vr_camera), P, P]
    lib.vr_last_error.argtypes = [P]
    lib.vr_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("vr_destroy", "vr_last_error", "vr_server_destroy", "vr_codec_destroy",
                        "vr_codec_param_count", "vr_codec_brick_count", "vr_codec_brick_size"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def _check(ctx, rc: int):
    if rc != VR_OK:
        msg = _lib.vr_last_error(ctx).decode() if ctx else ""
        raise VRError(rc, msg)


def make_camera(cam: dict) -> vr_camera:
    c = vr_camera()
    c.eye[:] = cam["eye"]
    c.target[:] = cam["target"]
    c.up[:] = cam["up"]
    c.fovy_deg = cam["fovy_deg"]
    c.width = cam["width"]
    c.height = cam["height"]
    c.step = cam["step"]
    c.term_alpha = cam["term_alpha"]
    return c


def _ptr(buf):
    """(address, keep-alive) of a numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data, buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), buf
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------- C-ABI calls

def vr_create(device: int = 0):
    h = ctypes.c_void_p()
    rc = _lib.vr_create(ctypes.byref(h), device)
    _check(None, rc)
    return h


def vr_destroy(ctx) -> None:
    _lib.vr_destroy(ctx)


def vr_load_cube(ctx, cube) -> None:
    """cube: float32 (nz, ny, nx), numpy (host) or torch (host or device)."""
    if getattr(cube, "dtype", None) not in (np.float32,) and str(getattr(cube, "dtype", "")) != "torch.float32":
        raise TypeError("cube must be float32")
    nz, ny, nx = cube.shape
    addr, keep = _ptr(cube)
    _check(ctx, _lib.vr_load_cube(ctx, addr, nx, ny, nz))


def vr_load_cube_host(ctx, cube) -> None:
    """Out-of-core load: cube is a float32 (nz, ny, nx) host array that must stay
    alive and unchanged while the context uses it (the VolumeRenderer keeps a
    reference)."""
    if getattr(cube, "dtype", None) != np.float32 or not isinstance(cube, np.ndarray):
        raise TypeError("cube must be a float32 numpy array")
    nz, ny, nx = cube.shape
    addr, keep = _ptr(cube)
    _check(ctx, _lib.vr_load_cube_host(ctx, addr, nx, ny, nz))


# int provider(void* user, const int64_t origin[3], const int32_t extent[3], float* dst,
#              int64_t row_stride, int64_t slice_stride)
BLOCK_PROVIDER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                  ctypes.c_int64, ctypes.c_int64)


def block_provider(provider):
    """(fn, user, keep) for the C ABI from either a native provider (an object
    with integer ``fn`` and ``user`` addresses, e.g. ``synth.BlockSource``) or a
    Python callable ``provider(origin_xyz, extent_xyz) -> float32 (ez, ey, ex)``
    (any thread may call it; an exception or a wrong shape reports a failure).
    Keep ``keep`` alive while the library may call the provider."""
    if hasattr(provider, "fn") and hasattr(provider, "user"):
        return provider.fn, provider.user, provider
    if not callable(provider):
        raise TypeError("provider must be callable or have native fn/user addresses")

    def cb(user, origin, extent, dst, row, slc):
        try:
            o = (int(origin[0]), int(origin[1]), int(origin[2]))
            e = (int(extent[0]), int(extent[1]), int(extent[2]))
            blk = np.asarray(provider(o, e), dtype=np.float32)
            if blk.shape != (e[2], e[1], e[0]):
                return 1
            n = (e[2] - 1) * slc + (e[1] - 1) * row + e[0]
            buf = np.ctypeslib.as_array(dst, shape=(n,))
            view = np.lib.stride_tricks.as_strided(buf, shape=(e[2], e[1], e[0]), strides=(slc * 4, row * 4, 4))
            view[...] = blk
            return 0
        except Exception:
            return 1

    f = BLOCK_PROVIDER(cb)
    return ctypes.cast(f, ctypes.c_void_p).value, None, f


def vr_load_cube_provider(ctx, provider, shape_xyz):
    """Out-of-core load from a brick provider (see ``block_provider``); returns
    the object to keep alive while the context uses the provider."""
    fn, user, keep = block_provider(provider)
    nx, ny, nz = (int(v) for v in shape_xyz)
    _check(ctx, _lib.vr_load_cube_provider(ctx, fn, user, nx, ny, nz))
    return keep


def vr_brick(ctx, bx: int, by: int, bz: int) -> None:
    _check(ctx, _lib.vr_brick(ctx, bx, by, bz))


def vr_set_transfer_function(ctx, points) -> None:
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 5)
    _check(ctx, _lib.vr_set_transfer_function(ctx, pts.ctypes.data, len(pts)))


def vr_set_camera(ctx, cam: dict) -> None:
    c = make_camera(cam)
    _check(ctx, _lib.vr_set_camera(ctx, ctypes.byref(c)))


def _mat16(m):
    """A 4x4 matrix (numpy, row r column c) as OpenGL's column-major 16 doubles."""
    a = np.asarray(m, dtype=np.float64)
    if a.shape == (4, 4):
        a = a.T
    return np.ascontiguousarray(a.reshape(16), dtype=np.float64)


def vr_camera_from_matrices(view, proj, width: int, height: int, step: float = 0.5,
                            term_alpha: float = 0.99) -> dict:
    """The camera dict equivalent to an OpenGL modelview and projection matrix
    (4x4 arrays, row r column c, or 16 column-major values)."""
    v, p = _mat16(view), _mat16(proj)
    cam = vr_camera()
    rc = _lib.vr_camera_from_matrices(v.ctypes.data, p.ctypes.data, int(width), int(height), float(step),
                                      float(term_alpha), ctypes.byref(cam))
    if rc != VR_OK:
        raise VRError(rc, "vr_camera_from_matrices")
    return {"eye": tuple(cam.eye), "target": tuple(cam.target), "up": tuple(cam.up), "fovy_deg": cam.fovy_deg,
            "width": cam.width, "height": cam.height, "step": cam.step, "term_alpha": cam.term_alpha}


def vr_set_camera_matrices(ctx, view, proj, width: int, height: int, step: float = 0.5,
                           term_alpha: float = 0.99) -> None:
    v, p = _mat16(view), _mat16(proj)
    _check(ctx, _lib.vr_set_camera_matrices(ctx, v.ctypes.data, p.ctypes.data, int(width), int(height),
                                            float(step), float(term_alpha)))


def vr_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, _lib.vr_set_option(ctx, option, int(value)))


def vr_render(ctx, out, stream=None) -> None:
    """Render into ``out`` (float32 (H, W, 4)): a CUDA tensor is written
    asynchronously on ``stream`` (default: torch's current stream); a numpy
    array or CPU tensor is filled synchronously."""
    addr, keep = _ptr(out)
    on_device = hasattr(out, "is_cuda") and out.is_cuda
    _check(ctx, _lib.vr_render(ctx, addr, _stream_handle(stream) if on_device else None))


def vr_get_stats(ctx) -> dict:
    s = vr_stats()
    _check(ctx, _lib.vr_get_stats(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in vr_stats._fields_ if name != "reserved"}


def vr_reset_stats(ctx) -> None:
    _check(ctx, _lib.vr_reset_stats(ctx))


def vr_get_brick_minmax(ctx, n_bricks: int) -> np.ndarray:
    out = np.zeros((n_bricks, 2), dtype=np.float32)
    _check(ctx, _lib.vr_get_brick_minmax(ctx, out.ctypes.data, n_bricks))
    return out


def vr_plan_brick_rects(cam: dict, shape_xyz, brick) -> np.ndarray:
    """Host-only: rendering rectangle (x0, y0, x1, y1) of every brick."""
    nb = [(n - 1 + b - 1) // b for n, b in zip(shape_xyz, brick)]
    n_bricks = nb[0] * nb[1] * nb[2]
    rects = np.zeros((n_bricks, 4), dtype=np.int32)
    c = make_camera(cam)
    rc = _lib.vr_plan_brick_rects(ctypes.byref(c), *shape_xyz, *brick, rects.ctypes.data, n_bricks)
    if rc != VR_OK:
        raise VRError(rc, "vr_plan_brick_rects rejected its arguments")
    return rects


def vr_plan_brick_tiles(cam: dict, shape_xyz, brick) -> np.ndarray:
    """Host-only: bool (n_bricks, n_tiles) of the (brick, 8x8 tile) items the
    planner emits (tiles row-major)."""
    nb = [(n - 1 + b - 1) // b for n, b in zip(shape_xyz, brick)]
    n_bricks = nb[0] * nb[1] * nb[2]
    n_tiles = ((cam["width"] + 7) // 8) * ((cam["height"] + 7) // 8)
    mask = np.zeros((n_bricks, n_tiles), dtype=np.uint8)
    c = make_camera(cam)
    rc = _lib.vr_plan_brick_tiles(ctypes.byref(c), *shape_xyz, *brick, mask.ctypes.data, n_bricks, n_tiles)
    if rc != VR_OK:
        raise VRError(rc, "vr_plan_brick_tiles rejected its arguments")
    return mask.astype(bool)


def _i32(v, n):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(-1))
    if a.size != n:
        raise ValueError(f"expected {n} integers")
    return a


def vr_kd_partition(shape_xyz, brick, n_parts: int) -> np.ndarray:
    """Host-only: int32 (n_parts, 6) brick ranges (lo xyz, hi xyz) of the k-d leaves."""
    B = _i32(brick, 3)
    out = np.zeros((n_parts, 6), dtype=np.int32)
    rc = _lib.vr_kd_partition(*shape_xyz, B.ctypes.data, int(n_parts), out.ctypes.data)
    if rc != VR_OK:
        raise VRError(rc, "vr_kd_partition rejected its arguments")
    return out


def vr_kd_order(shape_xyz, brick, n_parts: int, eye) -> np.ndarray:
    """Host-only: leaf numbers front to back as seen from ``eye``."""
    B = _i32(brick, 3)
    e = np.ascontiguousarray(np.asarray(eye, dtype=np.float64).reshape(3))
    out = np.zeros(n_parts, dtype=np.int32)
    rc = _lib.vr_kd_order(*shape_xyz, B.ctypes.data, int(n_parts), e.ctypes.data, out.ctypes.data)
    if rc != VR_OK:
        raise VRError(rc, "vr_kd_order rejected its arguments")
    return out


def vr_set_region(ctx, lo, hi) -> None:
    lo_, hi_ = _i32(lo, 3), _i32(hi, 3)
    _check(ctx, _lib.vr_set_region(ctx, lo_.ctypes.data, hi_.ctypes.data))


def vr_region_rect(ctx) -> np.ndarray:
    r = np.zeros(4, dtype=np.int32)
    _check(ctx, _lib.vr_region_rect(ctx, r.ctypes.data))
    return r


def vr_plan_region_rect(cam: dict, shape_xyz, brick, lo, hi) -> np.ndarray:
    """Host-only: rendering rectangle (x0, y0, x1, y1) of the brick range [lo, hi)."""
    B, lo_, hi_ = _i32(brick, 3), _i32(lo, 3), _i32(hi, 3)
    r = np.zeros(4, dtype=np.int32)
    c = make_camera(cam)
    rc = _lib.vr_plan_region_rect(ctypes.byref(c), *shape_xyz, B.ctypes.data, lo_.ctypes.data,
                                  hi_.ctypes.data, r.ctypes.data)
    if rc != VR_OK:
        raise VRError(rc, "vr_plan_region_rect rejected its arguments")
    return r


def vr_render_rect(ctx, rect, out, stream=None) -> None:
    """Render only the pixels of ``rect`` into ``out`` (float32 (rows, cols, 4))."""
    r = _i32(rect, 4)
    addr, keep = _ptr(out)
    on_device = hasattr(out, "is_cuda") and out.is_cuda
    _check(ctx, _lib.vr_render_rect(ctx, r.ctypes.data, addr, _stream_handle(stream) if on_device else None))


def vr_composite_subimages(ctx, images, rects, out, stream=None) -> None:
    """Front-to-back 'over' fold of sub-images (CUDA tensors, or None for an empty
    rect) with their rects into ``out`` (float32 (H, W, 4))."""
    n = len(images)
    ptrs = (ctypes.c_void_p * max(n, 1))()
    keep = []
    for k, im in enumerate(images):
        if im is None:
            ptrs[k] = None
            continue
        a, kk = _ptr(im)
        ptrs[k] = a
        keep.append(kk)
    R = np.ascontiguousarray(np.asarray(rects, dtype=np.int32).reshape(n, 4)) if n else np.zeros((1, 4), np.int32)
    addr, keep_out = _ptr(out)
    on_device = hasattr(out, "is_cuda") and out.is_cuda
    _check(ctx, _lib.vr_composite_subimages(ctx, n, ctypes.cast(ptrs, ctypes.c_void_p), R.ctypes.data, addr,
                                            _stream_handle(stream) if on_device else None))


def vr_server_create(ctx, arena_bytes: int, max_batch: int = 64):
    h = ctypes.c_void_p()
    _check(ctx, _lib.vr_server_create(ctx, int(arena_bytes), int(max_batch), ctypes.byref(h)))
    return h


def vr_server_submit(srv, ctx, cam: dict, out, tf=None) -> int:
    """Queue a frame into ``out`` (CUDA float32 (H, W, 4)); ``tf`` None keeps the
    transfer function in force.  Returns the ticket.  ``ctx`` is the served
    context (for error messages)."""
    c = make_camera(cam)
    addr, keep = _ptr(out)
    t = ctypes.c_int64()
    if tf is None:
        rc = _lib.vr_server_submit(srv, ctypes.byref(c), None, 0, addr, ctypes.byref(t))
    else:
        pts = np.ascontiguousarray(tf, dtype=np.float64).reshape(-1, 5)
        rc = _lib.vr_server_submit(srv, ctypes.byref(c), pts.ctypes.data, len(pts), addr, ctypes.byref(t))
    _check(ctx, rc)
    return t.value


def vr_server_wait(srv, ctx, ticket: int, timeout_s: float = -1.0) -> float:
    """Wait for a request; returns its latency in ms (submission to completion)."""
    lat = ctypes.c_double()
    rc = _lib.vr_server_wait(srv, int(ticket), float(timeout_s), ctypes.byref(lat))
    if rc != VR_OK:
        raise VRError(rc, f"request {ticket} failed")
    return lat.value


def vr_server_get_stats(srv) -> dict:
    s = vr_server_stats()
    rc = _lib.vr_server_get_stats(srv, ctypes.byref(s))
    if rc != VR_OK:
        raise VRError(rc, "vr_server_get_stats")
    return {name: getattr(s, name) for name, _ in vr_server_stats._fields_}


def vr_server_destroy(srv) -> None:
    _lib.vr_server_destroy(srv)


def to_bf16_bits(x) -> np.ndarray:
    """float32 values -> BF16 bit patterns (uint16), round to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_float(h) -> np.ndarray:
    return (np.asarray(h, dtype=np.uint32) << 16).view(np.float32)


def vr_codec_gemm_check(a_bf16, b_bf16, a_mn_major=0, b_mn_major=0) -> np.ndarray:
    """D = A B^T on the tensor cores (diagnostic): A (128, K), B (N, K) BF16 bits."""
    A = np.ascontiguousarray(a_bf16, dtype=np.uint16)
    B = np.ascontiguousarray(b_bf16, dtype=np.uint16)
    K, N = A.shape[1], B.shape[0]
    D = np.zeros((128, N), dtype=np.float32)
    rc = _lib.vr_codec_gemm_check(A.ctypes.data, B.ctypes.data, K, N, int(a_mn_major), int(b_mn_major),
                                  D.ctypes.data)
    if rc != VR_OK:
        raise VRError(rc, "vr_codec_gemm_check")
    return D


class Codec:
    """Learned brick codec (see include/vr.h): latents + shared MLP on the tensor cores."""

    HIDDEN, K_IN, LATENT, NODES = 64, 32, 16, 8

    def __init__(self, n_bricks: int, brick):
        h = ctypes.c_void_p()
        B = _i32(brick, 3)
        rc = _lib.vr_codec_create(int(n_bricks), B.ctypes.data, ctypes.byref(h))
        if rc != VR_OK:
            raise VRError(rc, "vr_codec_create")
        self.h, self.n_bricks, self.brick = h, int(n_bricks), tuple(int(b) for b in brick)
        self.n_params = int(_lib.vr_codec_param_count(h))

    def close(self):
        if self.h:
            _lib.vr_codec_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _rc(self, rc, what):
        if rc != VR_OK:
            raise VRError(rc, what)

    # parameter vector <-> dict of arrays (layout of include/vr.h)
    def pack(self, p: dict, lat) -> np.ndarray:
        parts = [np.asarray(p["W1"], np.float32).reshape(-1), np.asarray(p["b1"], np.float32).reshape(-1),
                 np.asarray(p["W2"], np.float32).reshape(-1), np.asarray(p["b2"], np.float32).reshape(-1),
                 np.asarray(p["w3"], np.float32).reshape(-1), np.asarray(p["b3"], np.float32).reshape(-1),
                 np.asarray(lat, np.float32).reshape(-1)]
        th = np.concatenate(parts)
        assert th.size == self.n_params
        return th

    def unpack(self, th) -> dict:
        H, K = self.HIDDEN, self.K_IN
        o = 0
        out = {}
        for name, shape in (("W1", (H, K)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
            n = int(np.prod(shape))
            out[name] = np.asarray(th[o:o + n]).reshape(shape)
            o += n
        out["lat"] = np.asarray(th[o:]).reshape(self.n_bricks, 8, 8, 8, 16)
        return out

    def set_params(self, theta, m, s):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        mm = np.ascontiguousarray(m, dtype=np.float32)
        ss = np.ascontiguousarray(s, dtype=np.float32)
        self._rc(_lib.vr_codec_set_params(self.h, th.ctypes.data, mm.ctypes.data, ss.ctypes.data),
                 "vr_codec_set_params")

    def get_params(self):
        th = np.zeros(self.n_params, np.float32)
        m = np.zeros(self.n_bricks, np.float32)
        s = np.zeros(self.n_bricks, np.float32)
        self._rc(_lib.vr_codec_get_params(self.h, th.ctypes.data, m.ctypes.data, s.ctypes.data), "vr_codec_get_params")
        return th, m, s

    @staticmethod
    def points(bricks, u) -> np.ndarray:
        """float32 (n, 4) point records: u (n, 3) local positions, brick index bits."""
        pts = np.zeros((len(bricks), 4), np.float32)
        pts[:, :3] = u
        pts[:, 3] = np.asarray(bricks, np.int32).view(np.float32)
        return pts

    def forward(self, pts) -> np.ndarray:
        pts = np.ascontiguousarray(pts, np.float32)
        out = np.zeros(len(pts), np.float32)
        self._rc(_lib.vr_codec_forward(self.h, pts.ctypes.data, len(pts), out.ctypes.data), "vr_codec_forward")
        return out

    def gradient(self, pts, targets):
        pts = np.ascontiguousarray(pts, np.float32)
        t = np.ascontiguousarray(targets, np.float32)
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._rc(_lib.vr_codec_gradient(self.h, pts.ctypes.data, t.ctypes.data, len(pts), g.ctypes.data,
                                        ctypes.byref(loss)), "vr_codec_gradient")
        return loss.value, g

    def fit_stats(self, cube_dev, floor=-3.4e38):
        nz, ny, nx = cube_dev.shape
        self._rc(_lib.vr_codec_fit_stats(self.h, cube_dev.data_ptr(), nx, ny, nz, float(floor)),
                 "vr_codec_fit_stats")

    def minmax(self) -> np.ndarray:
        out = np.zeros((self.n_bricks, 2), np.float32)
        self._rc(_lib.vr_codec_get_minmax(self.h, out.ctypes.data), "vr_codec_get_minmax")
        return out

    def train(self, cube_dev, steps: int, batch: int, lr: float, seed: int = 1, active_frac: float = 0.0) -> float:
        nz, ny, nx = cube_dev.shape
        loss = ctypes.c_double()
        self._rc(_lib.vr_codec_train(self.h, cube_dev.data_ptr(), nx, ny, nz, int(steps), int(batch), float(lr),
                                     float(active_frac), int(seed), ctypes.byref(loss)), "vr_codec_train")
        return loss.value

    def _slab_args(self, slab_dev, shape_xyz, bz0, bz1):
        nx, ny, nz = (int(v) for v in shape_xyz)
        bz = self.brick[2]
        planes = min(bz1 * bz, nz - 1) - bz0 * bz + 1
        if tuple(slab_dev.shape) != (planes, ny, nx) or not slab_dev.is_contiguous():
            raise ValueError(f"slab must be a contiguous ({planes}, {ny}, {nx}) device tensor")
        return slab_dev.data_ptr(), nx, ny, nz, int(bz0), int(bz1)

    def fit_stats_slab(self, slab_dev, shape_xyz, bz0: int, bz1: int, floor=-3.4e38):
        """fit_stats for the bricks of layers [bz0, bz1) from the slab of the cube's
        planes bz0*Bz .. min(bz1*Bz, nz-1)."""
        self._rc(_lib.vr_codec_fit_stats_slab(self.h, *self._slab_args(slab_dev, shape_xyz, bz0, bz1), float(floor)),
                 "vr_codec_fit_stats_slab")

    def train_slab(self, slab_dev, shape_xyz, bz0: int, bz1: int, steps: int, batch: int, lr: float,
                   mlp_lr: float = None, seed: int = 1) -> float:
        """Adam steps on the slab's bricks: their latents at lr, the shared network
        at mlp_lr (default lr; 0 keeps it)."""
        loss = ctypes.c_double()
        self._rc(_lib.vr_codec_train_slab(self.h, *self._slab_args(slab_dev, shape_xyz, bz0, bz1), int(steps),
                                          int(batch), float(lr), float(lr if mlp_lr is None else mlp_lr), int(seed),
                                          ctypes.byref(loss)), "vr_codec_train_slab")
        return loss.value

    def decode_bricks(self, bricks_dev, out_dev, slots_dev=None, stream=None):
        self._rc(_lib.vr_codec_decode_bricks(self.h, bricks_dev.data_ptr(),
                                             None if slots_dev is None else slots_dev.data_ptr(),
                                             int(bricks_dev.numel()), out_dev.data_ptr(), _stream_handle(stream)),
                 "vr_codec_decode_bricks")


class Server:
    """A serving loop on a VolumeRenderer (which it owns until closed)."""

    def __init__(self, renderer, arena_bytes: int, max_batch: int = 64):
        self.r = renderer
        self.h = vr_server_create(renderer.ctx, arena_bytes, max_batch)

    def submit(self, cam: dict, out, tf=None) -> int:
        return vr_server_submit(self.h, self.r.ctx, cam, out, tf)

    def wait(self, ticket: int, timeout_s: float = -1.0) -> float:
        return vr_server_wait(self.h, self.r.ctx, ticket, timeout_s)

    def stats(self) -> dict:
        return vr_server_get_stats(self.h)

    def close(self):
        if self.h:
            vr_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def vr_render_noalloc(cube, brick, points, cam: dict, out, stream=None) -> None:
    """Allocation-free render: ``cube`` and ``out`` are float32 CUDA tensors of
    shapes (nz, ny, nx) and (H, W, 4) on the current device; scratch lives in
    the library's static device array, so calls that overlap on the GPU race.
    Raises ValueError for any other shape, dtype or device before calling the
    library (the library reads and writes by the sizes it is given)."""
    import torch
    for name, t in (("cube", cube), ("out", out)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
            raise ValueError(f"{name} must be a float32 torch tensor")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device")
    if cube.dim() != 3:
        raise ValueError("cube must have shape (nz, ny, nx)")
    if tuple(out.shape) != (int(cam["height"]), int(cam["width"]), 4):
        raise ValueError(f"out must have shape ({cam['height']}, {cam['width']}, 4)")
    nz, ny, nx = cube.shape
    caddr, ckeep = _ptr(cube)
    oaddr, okeep = _ptr(out)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 5)
    c = make_camera(cam)
    rc = _lib.vr_render_noalloc(caddr, nx, ny, nz, *brick, pts.ctypes.data, len(pts),
                                ctypes.byref(c), oaddr, _stream_handle(stream))
    if rc != VR_OK:
        raise VRError(rc, "vr_render_noalloc failed")


def vr_last_error(ctx) -> str:
    return _lib.vr_last_error(ctx).decode()


# ------------------------------------------------------------------ convenience

class VolumeRenderer:
    """Owns one context; methods call the entry points above."""

    def __init__(self, device: int = 0):
        self.ctx = vr_create(device)
        self.shape_xyz = None
        self.brick_size = None
        self.camera = None

    def close(self):
        if self.ctx:
            vr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_cube(self, cube):
        vr_load_cube(self.ctx, cube)
        nz, ny, nx = cube.shape
        self.shape_xyz = (nx, ny, nz)
        self._host_cube = None

    def load_cube_codec(self, codec, shape_xyz):
        """Render from a learned codec (bricks decoded into the device cache)."""
        _check(self.ctx, _lib.vr_load_cube_codec(self.ctx, codec.h, *shape_xyz))
        self.shape_xyz = tuple(int(v) for v in shape_xyz)
        self._host_cube = codec

    def set_codec_fallback(self, cube, bound, floor=-3.4e38):
        """Bricks of a learned context whose decode error exceeds `bound` are copied
        from the plain host cube (float32 (nz, ny, nx), kept referenced until the
        next brick()) instead of decoded; cube=None turns the fallback off."""
        if cube is None:
            _check(self.ctx, _lib.vr_set_codec_fallback(self.ctx, None, float(bound), float(floor)))
            self._fallback_cube = None
            return
        if not isinstance(cube, np.ndarray) or cube.dtype != np.float32 or not cube.flags.c_contiguous:
            raise TypeError("cube must be a C-contiguous float32 numpy array")
        if tuple(cube.shape[::-1]) != tuple(self.shape_xyz):
            raise ValueError("the cube's shape differs from the learned context's")
        _check(self.ctx, _lib.vr_set_codec_fallback(self.ctx, cube.ctypes.data, float(bound), float(floor)))
        self._fallback_cube = cube

    def set_codec_fallback_provider(self, provider, bound, floor=-3.4e38):
        """As set_codec_fallback, with the plain blocks from a brick provider
        (see ``block_provider``; used during the next brick() only)."""
        if provider is None:
            _check(self.ctx, _lib.vr_set_codec_fallback_provider(self.ctx, None, None, float(bound), float(floor)))
            self._fallback_cube = None
            return
        fn, user, keep = block_provider(provider)
        _check(self.ctx, _lib.vr_set_codec_fallback_provider(self.ctx, fn, user, float(bound), float(floor)))
        self._fallback_cube = keep

    def codec_brick_errors(self):
        """(per-brick decode errors, number of bricks that fall back) of the last brick()."""
        err = np.zeros(self.n_bricks, dtype=np.float32)
        n = ctypes.c_int64(0)
        _check(self.ctx, _lib.vr_codec_brick_errors(self.ctx, err.ctypes.data, ctypes.byref(n)))
        return err, int(n.value)

    def load_cube_host(self, cube):
        """Out-of-core: the cube stays in host memory (a reference is kept)."""
        cube = np.ascontiguousarray(cube, dtype=np.float32)
        vr_load_cube_host(self.ctx, cube)
        nz, ny, nx = cube.shape
        self.shape_xyz = (nx, ny, nz)
        self._host_cube = cube

    def load_cube_provider(self, provider, shape_xyz):
        """Out-of-core from a brick provider (see ``block_provider``): no host
        copy of the cube is kept; bricks are requested as frames need them."""
        self._host_cube = vr_load_cube_provider(self.ctx, provider, shape_xyz)
        self.shape_xyz = tuple(int(v) for v in shape_xyz)

    def brick(self, bx, by, bz):
        vr_brick(self.ctx, bx, by, bz)
        self.brick_size = (bx, by, bz)

    @property
    def n_bricks(self):
        nb = [(n - 1 + b - 1) // b for n, b in zip(self.shape_xyz, self.brick_size)]
        return nb[0] * nb[1] * nb[2]

    def set_transfer_function(self, tf):
        vr_set_transfer_function(self.ctx, tf)

    def set_camera(self, cam):
        vr_set_camera(self.ctx, cam)
        self.camera = dict(cam)

    def set_camera_matrices(self, view, proj, width, height, step=0.5, term_alpha=0.99):
        """Camera from the viewer's OpenGL modelview and projection matrices."""
        vr_set_camera_matrices(self.ctx, view, proj, width, height, step, term_alpha)
        self.camera = vr_camera_from_matrices(view, proj, width, height, step, term_alpha)

    def set_option(self, option, value):
        vr_set_option(self.ctx, option, value)

    def render(self, out=None, stream=None):
        """Render one frame; returns ``out`` (allocates a CUDA tensor if None)."""
        if out is None:
            import torch
            out = torch.empty((self.camera["height"], self.camera["width"], 4),
                              dtype=torch.float32, device="cuda")
        vr_render(self.ctx, out, stream)
        return out

    def stats(self):
        return vr_get_stats(self.ctx)

    def reset_stats(self):
        vr_reset_stats(self.ctx)

    def brick_minmax(self):
        return vr_get_brick_minmax(self.ctx, self.n_bricks)

    def set_region(self, lo, hi):
        vr_set_region(self.ctx, lo, hi)

    def region_rect(self):
        return vr_region_rect(self.ctx)

    def render_rect(self, rect, out=None, stream=None):
        """Render the pixels of ``rect``; returns ``out`` (allocates a CUDA tensor
        of the rect's size if None; None for an empty rect)."""
        x0, y0, x1, y1 = (int(v) for v in rect)
        if x1 < x0 or y1 < y0:
            return None
        if out is None:
            import torch
            out = torch.empty((y1 - y0 + 1, x1 - x0 + 1, 4), dtype=torch.float32, device="cuda")
        vr_render_rect(self.ctx, rect, out, stream)
        return out

    def composite(self, images, rects, out=None, stream=None):
        """Root fold of sub-images (front to back) into a full frame."""
        if out is None:
            import torch
            out = torch.empty((self.camera["height"], self.camera["width"], 4),
                              dtype=torch.float32, device="cuda")
        vr_composite_subimages(self.ctx, images, rects, out, stream)
        return out
