"""Arbitrary-precision brute-force ray caster -- TEST INFRASTRUCTURE.

An independent restatement of the same readings as ``vr_oracle.c`` (Sections
1.2, 2.3.2 and 2.3.3 of arXiv:1205.0282), written differently on purpose so
that a slip in either one shows up as a disagreement:

* entry/exit by clipping the ray against the six faces of the domain one
  half-space at a time (instead of a per-axis slab min/max);
* tri-linear interpolation as the tensor-product sum over the 8 corners
  (instead of nested lerps);
* the transfer function by scanning for the last control point at or below v;
* compositing in closed product form: a run's colour is
  sum_k alpha_k c_k prod_{j<k} (1 - alpha_j) and its opacity
  1 - prod_k (1 - alpha_k), cut after the first sample whose opacity reaches
  the limit; runs are folded the same way with their own opacities.

All arithmetic is mpmath at 50 significant digits.  It is slow: use it on
cubes of a few voxels and images of a few dozen pixels.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 50


def _vec(v):
    return [mp.mpf(float(x)) for x in v]


def _norm(v):
    n = mp.sqrt(sum(x * x for x in v))
    return [x / n for x in v]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _clip(eye, d, ext):
    """Parametric interval of the line eye + t d inside [0, ext] (all axes)."""
    t_in, t_out = mp.mpf("-inf"), mp.mpf("inf")
    for a in range(3):
        for bound, outward in ((mp.mpf(0), -1), (mp.mpf(ext[a]), 1)):
            # half-space: outward * (x_a - bound) <= 0
            num = outward * (eye[a] - bound)
            den = outward * d[a]
            if den == 0:
                if num > 0:
                    return None
                continue
            t = -num / den
            if den < 0:
                t_in = max(t_in, t)   # entering this half-space
            else:
                t_out = min(t_out, t)
    return t_in, t_out


def _value(cube, p):
    nz, ny, nx = cube.shape
    n = (nx, ny, nz)
    i0, f = [], []
    for a in range(3):
        q = min(max(p[a], mp.mpf(0)), mp.mpf(n[a] - 1))
        i = int(mp.floor(q))
        i = min(i, n[a] - 2)
        i0.append(i)
        f.append(q - i)
    total = mp.mpf(0)
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                w = ((f[0] if cx else 1 - f[0]) * (f[1] if cy else 1 - f[1]) *
                     (f[2] if cz else 1 - f[2]))
                total += w * mp.mpf(float(cube[i0[2] + cz, i0[1] + cy, i0[0] + cx]))
    return total


def _tf(tf, v):
    rows = [[mp.mpf(float(x)) for x in r] for r in tf]
    if v <= rows[0][0]:
        return rows[0][1:]
    if v >= rows[-1][0]:
        return rows[-1][1:]
    s = max(k for k in range(len(rows)) if rows[k][0] <= v)
    lo, hi = rows[s], rows[s + 1]
    w = (v - lo[0]) / (hi[0] - lo[0])
    return [lo[c] + w * (hi[c] - lo[c]) for c in range(1, 5)]


def _composite(items, tau):
    """items: list of (colour[3], opacity).  Product-form front-to-back sum cut
    after the first item whose accumulated opacity reaches tau.  Returns
    (rgba, list of accumulated opacities seen at each step)."""
    trans = mp.mpf(1)
    rgb = [mp.mpf(0)] * 3
    seen = []
    for col, op in items:
        for c in range(3):
            rgb[c] += trans * col[c]
        trans *= (1 - op)
        acc = 1 - trans
        seen.append(acc)
        if acc >= tau:
            break
    return rgb + [1 - trans], seen


def ray(cube, tf, cam, i, j, brick=None, amb_alpha=1e-5, amb_steps=1e-4):
    """(rgba as 4 mpf, ambiguous flag bits) for pixel (i, j)."""
    nz, ny, nx = cube.shape
    ext = (nx - 1, ny - 1, nz - 1)
    eye, tgt, up = _vec(cam["eye"]), _vec(cam["target"]), _vec(cam["up"])
    W, H = cam["width"], cam["height"]
    f = _norm([tgt[a] - eye[a] for a in range(3)])
    r = _norm(_cross(f, up))
    u = _cross(r, f)
    th = mp.tan(mp.mpf(cam["fovy_deg"]) * mp.pi / 360)
    qx = (mp.mpf(2) * (i + mp.mpf("0.5")) / W - 1) * th * mp.mpf(W) / H
    qy = (1 - mp.mpf(2) * (j + mp.mpf("0.5")) / H) * th
    d = _norm([f[a] + qx * r[a] + qy * u[a] for a in range(3)])
    zero = [mp.mpf(0)] * 4
    span = _clip(eye, d, ext)
    if span is None:
        return zero, 0
    t0, t1 = max(span[0], mp.mpf(0)), span[1]
    if not (t1 > t0):
        return zero, 0
    L = t1 - t0
    dt = mp.mpf(cam["step"])
    tau = mp.mpf(cam["term_alpha"])
    amb = 0
    x = L / dt
    if abs(x - mp.nint(x)) < amb_steps:
        amb |= 1
    pe = [eye[a] + t0 * d[a] for a in range(3)]
    # samples and their owners
    runs = []   # list of (owner, [ (colour, alpha) ... ])
    nb = None
    if brick is not None:
        nb = [(e + b - 1) // b for e, b in zip(ext, brick)]
    k = 0
    while k * dt < L:
        p = [pe[a] + (k * dt) * d[a] for a in range(3)]
        if brick is None:
            owner = 0
        else:
            owner = tuple(min(int(mp.floor(min(max(p[a], 0), ext[a]) / brick[a])), nb[a] - 1)
                          for a in range(3))
        v = _value(cube, p)
        cr, cg, cb, a = _tf(tf, v)
        alpha = 1 - (1 - a) ** (dt / 1)
        item = ([alpha * cr, alpha * cg, alpha * cb], alpha)
        if not runs or runs[-1][0] != owner:
            runs.append((owner, []))
        runs[-1][1].append(item)
        k += 1
    segs = []
    for _, items in runs:
        rgba, seen = _composite(items, tau)
        if any(abs(s - tau) < amb_alpha for s in seen):
            amb |= 2
        segs.append((rgba[:3], rgba[3]))
    rgba, seen = _composite(segs, tau)
    if any(abs(s - tau) < amb_alpha for s in seen):
        amb |= 2
    return rgba, amb


def render(cube, tf, cam, brick=None, pixels=None, **kw):
    """Float64 (npix, 4) image (row-major pixel list or whole image) and flags."""
    W, H = cam["width"], cam["height"]
    if pixels is None:
        pixels = range(W * H)
    out, flags = [], []
    for pix in pixels:
        rgba, amb = ray(cube, tf, cam, int(pix) % W, int(pix) // W, brick, **kw)
        out.append([float(x) for x in rgba])
        flags.append(amb)
    return np.array(out, dtype=np.float64), np.array(flags, dtype=np.uint8)
