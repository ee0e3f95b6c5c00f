"""Sort-last distribution of one frame over ranks (Sections 2.3.1, 2.3.3 and
2.3.4 of arXiv:1205.0282).

Rank r owns leaf r of the k-d partition of the brick grid (``vr_kd_partition``),
renders the bricks of that leaf into a sub-image clipped to the leaf's rendering
rectangle (``vr_region_rect``, ``vr_render_rect``) and sends rectangle and
pixels straight to the root (direct send: the only data exchange of the path).
The root folds the sub-images front to back in the visibility order of the
leaves from the eye (``vr_kd_order``) with ``vr_composite_subimages``.

Only argument marshalling and the exchange live here; every pixel is computed
by ``libvr.so``.  The exchange uses ``torch.distributed`` point-to-point sends
(gloo for CPU tensors, NCCL for CUDA tensors); a rank that fails or leaves
before the exchange makes the root's receive raise (at once when its connection
closes, else after the exchange's timeout) instead of hanging.
"""
from __future__ import annotations

import numpy as np

from .vr import vr_kd_order, vr_kd_partition

_TAG_RECT, _TAG_PIXELS = 11, 12


def leaf_ranges(shape_xyz, brick, world: int) -> np.ndarray:
    """int32 (world, 6): brick ranges (lo xyz, hi xyz) of the ranks' leaves."""
    return vr_kd_partition(shape_xyz, brick, world)


def visibility_order(shape_xyz, brick, world: int, eye) -> np.ndarray:
    """Leaf (= rank) numbers front to back as seen from ``eye``."""
    return vr_kd_order(shape_xyz, brick, world, eye)


def exchange_subimages(dist, rank: int, world: int, rect, sub, root: int = 0, device="cpu",
                       timeout_s: float = 60.0):
    """Direct send of every rank's (rect, sub-image) to the root.

    rect: (x0, y0, x1, y1) inclusive, x1 < x0 for an empty sub-image; sub: float32
    tensor (y1-y0+1, x1-x0+1, 4) on ``device`` (None when empty).  Returns, on the
    root, a list indexed by rank of (rect as int32 numpy array, tensor or None);
    None elsewhere.  Every send and receive waits at most ``timeout_s`` seconds and
    raises RuntimeError after that, or as soon as the peer's connection closes.
    """
    import datetime

    import torch

    limit = datetime.timedelta(seconds=timeout_s)

    def send(t, tag):
        dist.isend(t, dst=root, tag=tag).wait(limit)

    def recv(t, src, tag):
        dist.irecv(t, src=src, tag=tag).wait(limit)

    r = torch.tensor([int(v) for v in rect], dtype=torch.int64, device=device)
    if rank != root:
        send(r, _TAG_RECT)
        if rect[2] >= rect[0] and rect[3] >= rect[1]:
            send(sub.contiguous().view(-1), _TAG_PIXELS)
        return None
    out = [None] * world
    out[root] = (np.asarray(rect, dtype=np.int32), sub if rect[2] >= rect[0] and rect[3] >= rect[1] else None)
    for src in range(world):
        if src == root:
            continue
        rr = torch.empty(4, dtype=torch.int64, device=device)
        recv(rr, src, _TAG_RECT)
        x0, y0, x1, y1 = (int(v) for v in rr.tolist())
        if x1 < x0 or y1 < y0:
            out[src] = (np.array([x0, y0, x1, y1], dtype=np.int32), None)
            continue
        buf = torch.empty((y1 - y0 + 1) * (x1 - x0 + 1) * 4, dtype=torch.float32, device=device)
        recv(buf, src, _TAG_PIXELS)
        out[src] = (np.array([x0, y0, x1, y1], dtype=np.int32), buf.view(y1 - y0 + 1, x1 - x0 + 1, 4))
    return out


def render_distributed(renderer, dist, rank: int, world: int, root: int = 0, stream=None):
    """One frame over ``world`` ranks: this rank renders its k-d leaf of the
    renderer's cube (which every rank holds) at the renderer's camera; the root
    returns the composited frame (a CUDA tensor), other ranks None.  The camera,
    transfer function, bricking and options must be the same on every rank."""
    import torch

    shape, brick, cam = renderer.shape_xyz, renderer.brick_size, renderer.camera
    ranges = leaf_ranges(shape, brick, world)
    renderer.set_region(ranges[rank, :3], ranges[rank, 3:])
    rect = renderer.region_rect()
    sub = renderer.render_rect(rect, stream=stream)
    torch.cuda.synchronize()
    on_gpu = dist.get_backend() == "nccl"
    payload = sub if (sub is None or on_gpu) else sub.cpu()
    got = exchange_subimages(dist, rank, world, rect, payload, root, "cuda" if on_gpu else "cpu")
    if rank != root:
        return None
    order = visibility_order(shape, brick, world, cam["eye"])
    images = [None if got[k][1] is None else got[k][1].cuda() for k in order]
    rects = np.stack([got[k][0] for k in order])
    return renderer.composite(images, rects, stream=stream)
