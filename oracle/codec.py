"""Learned brick codec, FP64 reference -- TEST INFRASTRUCTURE (oracle side).

Not in the paper (an extension that stores each brick as a small latent grid
decoded by a shared MLP).  Definition, used by the GPU kernels and restated here:

* Brick b has a latent grid L_b of 8 x 8 x 8 nodes x 16 channels.  A voxel at
  local position u in [0, B]^3 (voxels of the brick and its +1 apron) has the
  normalised position x = u / B and latent z = trilinear interpolation of L_b at
  g = 7 x (node spacing B / 7).
* Fourier features of x: for each axis a, sin(pi x_a), cos(pi x_a),
  sin(2 pi x_a), cos(2 pi x_a) -> 12 values.
* Input row: [z (16), Fourier (12), 0 (4)] -> 32 values.
* MLP: z1 = W1 in + b1 (64), h1 = silu(z1), z2 = W2 h1 + b2 (64),
  h2 = silu(z2), y = w3 . h2 + b3;  silu(t) = t / (1 + exp(-t)).
* Decoded value: v = y s_b + m_b (per-brick scale and offset).

The latent grid is held in BF16 (the values interpolated are the BF16 roundings
of the FP32 master latents that training updates), and the tensor-core kernels
take their operands in BF16 (round to nearest even):
the input row, W1, W2, w3, h1 (layer 2's input) and, in the backward pass, the
layer gradients g2 = dL/dz2 and g1 = dL/dz1 where they enter a product (the
bias gradients sum them unrounded).  With
``bf16=True`` this module rounds the same quantities at the same points, so the
GPU result differs from it by FP32 accumulation only; with ``bf16=False`` it is
the plain FP64 definition (used to pin the formulas by finite differences).

Loss of a training step over points P with targets t: mean over P of (v - t)^2.
"""
from __future__ import annotations

import numpy as np

LATENT = 16
NODES = 8
HIDDEN = 64
K_IN = 32


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(t):
    return t / (1.0 + np.exp(-t))


def silu_grad(t):
    s = 1.0 / (1.0 + np.exp(-t))
    return s * (1.0 + t * (1.0 - s))


def fourier(x):
    """x: (P, 3) in [0, 1] -> (P, 12)."""
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for a in range(3):
        cols += [np.sin(np.pi * x[:, a]), np.cos(np.pi * x[:, a]),
                 np.sin(2 * np.pi * x[:, a]), np.cos(2 * np.pi * x[:, a])]
    return np.stack(cols, axis=1)


def trilinear_weights(x):
    """Node indices (P, 8, 3) and weights (P, 8) of the trilinear interpolation
    at g = 7 x; corner c = (cx, cy, cz) bits (x fastest)."""
    g = np.asarray(x, dtype=np.float64) * (NODES - 1)
    i0 = np.clip(np.floor(g).astype(np.int64), 0, NODES - 2)
    f = g - i0
    idx = np.empty((len(g), 8, 3), dtype=np.int64)
    w = np.empty((len(g), 8))
    for c in range(8):
        bits = np.array([(c >> a) & 1 for a in range(3)])
        idx[:, c, :] = i0 + bits
        w[:, c] = np.prod(np.where(bits[None, :] == 1, f, 1.0 - f), axis=1)
    return idx, w


def latent_interp(lat, brick, x):
    """lat: (n_bricks, 8, 8, 8, 16) indexed [b][z][y][x][ch]; brick: (P,) ints."""
    idx, w = trilinear_weights(x)
    z = np.zeros((len(brick), LATENT))
    for c in range(8):
        node = lat[brick, idx[:, c, 2], idx[:, c, 1], idx[:, c, 0]]
        z += w[:, c:c + 1] * node
    return z


def input_rows(lat, brick, x, bf=True):
    z = latent_interp(bf16(lat) if bf else lat, brick, x)
    row = np.concatenate([z, fourier(x), np.zeros((len(brick), K_IN - LATENT - 12))], axis=1)
    return bf16(row) if bf else row


def forward(params, lat, brick, x, bf=True):
    """Returns (v, cache) for points (brick, x)."""
    W1, b1, W2, b2, w3, b3, m, s = (params[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3", "m", "s"))
    q = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    IN = input_rows(lat, brick, x, bf)
    z1 = IN @ q(W1).T + b1
    h1 = q(silu(z1))
    z2 = h1 @ q(W2).T + b2
    h2 = silu(z2)
    y = h2 @ q(w3) + b3
    v = y * s[brick] + m[brick]
    return v, dict(IN=IN, z1=z1, h1=h1, z2=z2, h2=h2, y=y)


def backward(params, lat, brick, x, target, bf=True, cache=None):
    """Loss mean((v - t)^2) and its gradients with respect to W1, b1, W2, b2, w3,
    b3 and the latent grid (same shape as lat).  If ``cache`` is a dict it
    receives the intermediate values (forward pass, dy, the layer gradients
    before and after rounding, dh1, din, the interpolation nodes and weights)."""
    W1, W2, w3, s = params["W1"], params["W2"], params["w3"], params["s"]
    q = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    v, c = forward(params, lat, brick, x, bf)
    P = len(brick)
    r = v - target
    loss = float(np.mean(r * r))
    dy = 2.0 * r * s[brick] / P
    g = {}
    g["b3"] = np.array(dy.sum())
    g["w3"] = c["h2"].T @ dy
    g2f = dy[:, None] * q(w3)[None, :] * silu_grad(c["z2"])
    g["b2"] = g2f.sum(axis=0)
    g2 = q(g2f)
    g["W2"] = g2.T @ c["h1"]
    dh1 = g2 @ q(W2)
    g1f = dh1 * silu_grad(c["z1"])
    g["b1"] = g1f.sum(axis=0)
    g1 = q(g1f)
    g["W1"] = g1.T @ c["IN"]
    din = g1 @ q(W1)
    dz = din[:, :LATENT]
    idx, w = trilinear_weights(x)
    dlat = np.zeros_like(lat, dtype=np.float64)
    for k in range(8):
        np.add.at(dlat, (brick, idx[:, k, 2], idx[:, k, 1], idx[:, k, 0]), w[:, k:k + 1] * dz)
    g["lat"] = dlat
    if cache is not None:
        cache.update(c)
        cache.update(v=v, dy=dy, g2f=g2f, g2=g2, dh1=dh1, g1f=g1f, g1=g1, din=din, idx=idx, w=w)
    return loss, g


def init_params(n_bricks, seed=0, brick_mean=None, brick_scale=None):
    """Seeded initialisation (uniform fan-in scaling; latents small)."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.uniform(-1, 1, (HIDDEN, K_IN)) / np.sqrt(28.0),
        "b1": np.zeros(HIDDEN),
        "W2": rng.uniform(-1, 1, (HIDDEN, HIDDEN)) / np.sqrt(HIDDEN),
        "b2": np.zeros(HIDDEN),
        "w3": rng.uniform(-1, 1, HIDDEN) / np.sqrt(HIDDEN),
        "b3": np.array(0.0),
        "m": np.zeros(n_bricks) if brick_mean is None else np.asarray(brick_mean, np.float64),
        "s": np.ones(n_bricks) if brick_scale is None else np.asarray(brick_scale, np.float64),
    }
    p["W1"][:, 28:] = 0.0
    lat = rng.normal(0.0, 0.1, (n_bricks, NODES, NODES, NODES, LATENT))
    return p, lat
