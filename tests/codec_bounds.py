"""Per-element error bounds of the learned codec's GPU arithmetic against the
FP64 codec oracle (test infrastructure).

The oracle (oracle/codec.py, bf16=True) rounds to BF16 at the same points as
the kernels, so a GPU value differs from the oracle's by two kinds of error:

* FP32 rounding of every other operation: products and sums on the CUDA
  cores, the tensor cores' FP32 accumulation, the hardware approximations in
  SiLU and its derivative, the Fourier features.  Each is bounded here by its
  textbook first-order model: a sum of n terms carries at most n units of
  roundoff times the sum of the magnitudes of the terms; the tensor cores are
  charged four FP32 ulps per K = 16 step (products are exact in FP32; the
  accumulation's internal alignment is not documented, so truncation is allowed);
  an approximate SiLU at (|t| + 8) 4 u relative (the exponential's argument t log2 e
  carries |t| u, ex2.approx and rcp.approx a few ulps each).
* A BF16 rounding decision that goes the other way: where the FP64 value lies
  within the GPU's error bound of a rounding boundary, the two rounded values
  may be one BF16 step apart.  Elsewhere they are equal (the error is absorbed
  by the rounding).  One step is allowed exactly at those elements.

Both propagate to the outputs through the layers with absolute values of the
weights and of the derivatives (first order).  The final bound is multiplied by
C = 2 for the second-order terms the first-order model drops.  Nothing here
computes a value the test compares: only magnitudes and error terms.
"""
from __future__ import annotations

import numpy as np

from oracle import codec as ref

U = 2.0 ** -24          # FP32 unit roundoff
U_ACC = 2.0 ** -23      # one FP32 ulp relative: a tensor-core accumulation step
C = 2.0                 # safety factor for second-order terms
AMPLIFY = 16.0          # see big_flip
TINY = 1e-30


def bf16_delta(pre, eps):
    """Largest difference between bf16(pre) and the BF16 rounding of any FP32
    value within eps of pre (0 where the rounding cannot change)."""
    pre = np.asarray(pre, dtype=np.float64)
    r0 = ref.bf16(pre)
    return np.maximum(np.abs(ref.bf16(pre + eps) - r0), np.abs(ref.bf16(pre - eps) - r0))


def big_flip(delta, eps):
    """Rounding decisions that may go the other way by a step much larger than
    the error that moves them (more than AMPLIFY times): the step then dominates
    every later error term.  Smaller steps (values near zero, whose BF16 steps are
    tiny) are simply carried by the bound."""
    return delta > AMPLIFY * eps


def _silu_parts(t):
    s = 1.0 / (1.0 + np.exp(-t))
    silu = t * s
    d1 = s * (1.0 + t * (1.0 - s))
    d2 = s * (1.0 - s) * (2.0 + t * (1.0 - 2.0 * s))
    return s, silu, d1, d2


def _silu_approx_err(t, value):
    return (np.abs(t) + 8.0) * 4.0 * U * np.abs(value) + TINY


TANH_REL = 2.0 ** -10.5   # hardware tanh.approx.f32: relative error about 2^-11, with margin


def _silu_fast_err(t, value):
    """silu(t) = h + h tanh(h), h = t / 2, with the hardware tanh (rendering
    decode): |h| times the tanh's relative error times |tanh(h)|, plus the
    roundings of h and of the FMA."""
    h = 0.5 * np.abs(t)
    return h * TANH_REL * np.abs(np.tanh(0.5 * t)) + 4.0 * U * np.abs(value) + TINY


def _tc_err(S, K):
    """Tensor-core product over K (FP32 accumulation, K / 16 steps)."""
    return 4.0 * (K / 16.0 + 1.0) * U_ACC * S


def _input_eps(latq, brick, x, B):
    """Bound on the GPU's error in the input row before its BF16 rounding.  The
    kernel forms x = u * fl(1 / B) (exact for a power-of-two B), g = 7 x, the
    interpolation fractions and weights (three roundings each) and eight FMAs;
    a lattice coordinate off by dg moves z by at most dg times its slope (the
    weight derivatives times |L|, or twice the brick's largest node where g is
    within dg of a node and the other cell may be used).  sincospif is within
    one ulp; the double angles add a few roundings."""
    P = len(brick)
    xB = np.asarray(x, dtype=np.float64)
    pow2 = np.array([b & (b - 1) == 0 for b in B])
    dx = np.where(pow2[None, :], 0.0, 2.0 * U * xB)
    g = xB * (ref.NODES - 1)
    dg = (ref.NODES - 1) * dx + U * g
    i0 = np.clip(np.floor(g), 0, ref.NODES - 2)
    fr = g - i0
    idx, w = ref.trilinear_weights(xB)
    absz = np.zeros((P, ref.LATENT))
    slope = np.zeros((P, ref.LATENT))
    for c in range(8):
        node = np.abs(latq[brick, idx[:, c, 2], idx[:, c, 1], idx[:, c, 0]])
        absz += w[:, c:c + 1] * node
        bits = [(c >> a) & 1 for a in range(3)]
        for a in range(3):
            dw = np.ones(P)
            for b in range(3):
                if b != a:
                    dw = dw * (fr[:, b] if bits[b] else 1.0 - fr[:, b])
            slope += (dg[:, a] * dw)[:, None] * node
    node_max = np.abs(latq).reshape(latq.shape[0], -1).max(axis=1)[brick]
    near = (np.abs(g - np.round(g)) <= dg).any(axis=1)
    eps = np.zeros((P, ref.K_IN))
    eps[:, :ref.LATENT] = 11.0 * U * absz + 2.0 * slope + np.where(near, 2.0 * node_max * dg.sum(axis=1), 0.0)[:, None]
    for a in range(3):
        sn, cs = np.sin(np.pi * xB[:, a]), np.cos(np.pi * xB[:, a])
        eps[:, ref.LATENT + 4 * a:ref.LATENT + 4 * a + 4] = \
            (8.0 * U * (np.abs(sn) + np.abs(cs)) ** 2 + 2.0 * np.pi * dx[:, a])[:, None]
    return eps


def forward_terms(p, lat, brick, x, B=(16, 16, 16), fast_silu=False):
    """Error terms of the forward pass (before the factor C): a dict with the
    per-point bound 'v' and the intermediate bounds the backward pass needs.
    Values come from the oracle's forward pass; only magnitudes and error terms
    are formed here.  x = u / B with u the FP32 positions the GPU was given;
    fast_silu: the SiLU of the rendering decode (hardware tanh)."""
    silu_err = _silu_fast_err if fast_silu else _silu_approx_err
    q = ref.bf16
    W1q, W2q, w3q = q(p["W1"]), q(p["W2"]), q(p["w3"])
    b1, b2, b3 = np.asarray(p["b1"]), np.asarray(p["b2"]), float(p["b3"])
    s, m = np.asarray(p["s"])[brick], np.asarray(p["m"])[brick]
    P = len(brick)
    v, fc = ref.forward(p, lat, brick, x, bf=True)
    latq = q(lat)
    idx, w = ref.trilinear_weights(x)
    eps_in = _input_eps(latq, brick, x, B)
    IN_pre = np.concatenate([ref.latent_interp(latq, brick, x), ref.fourier(x),
                             np.zeros((P, ref.K_IN - ref.LATENT - 12))], axis=1)
    IN = fc["IN"]
    dIN = bf16_delta(IN_pre, eps_in)
    # layer 1 (K = 32) and its SiLU, rounded to BF16 for layer 2
    z1 = fc["z1"]
    S1 = np.abs(IN) @ np.abs(W1q).T
    dz1 = dIN @ np.abs(W1q).T + _tc_err(S1, 32) + U * (np.abs(z1) + np.abs(b1))
    _, _, sg1, sgg1 = _silu_parts(z1)
    h1_pre = ref.silu(z1)
    eh1 = np.abs(sg1) * dz1 + silu_err(z1, h1_pre)
    h1 = fc["h1"]
    dh1 = bf16_delta(h1_pre, eh1)
    # layer 2 (K = 64), SiLU in FP32, the output unit on the CUDA cores
    z2 = fc["z2"]
    S2 = np.abs(h1) @ np.abs(W2q).T
    dz2 = dh1 @ np.abs(W2q).T + _tc_err(S2, 64) + U * (np.abs(z2) + np.abs(b2))
    _, _, sg2, sgg2 = _silu_parts(z2)
    h2 = fc["h2"]
    dh2 = np.abs(sg2) * dz2 + silu_err(z2, h2)
    y = fc["y"]
    Sy = np.abs(h2) @ np.abs(w3q) + abs(b3)
    dy_ = dh2 @ np.abs(w3q) + 2.0 * 34.0 * U * Sy
    dv = np.abs(s) * dy_ + U * (np.abs(y * s) + np.abs(m))
    return dict(v=dv, IN=IN, dIN=dIN, z1=z1, dz1=dz1, h1=h1, dh1=dh1, sg1=sg1, sgg1=sgg1,
                z2=z2, dz2=dz2, h2=h2, dh2=dh2, sg2=sg2, sgg2=sgg2, value=v, w=w, idx=idx,
                W1q=W1q, W2q=W2q, w3q=w3q, flips=int((dIN > 0).sum() + (dh1 > 0).sum()),
                ambiguous=big_flip(dIN, eps_in).any(axis=1) | big_flip(dh1, eh1).any(axis=1))


def forward_bound(p, lat, brick, x, B=(16, 16, 16), fast_silu=False):
    """Per-point bound on |v_gpu - v_oracle| (bf16=True)."""
    return C * forward_terms(p, lat, brick, x, B, fast_silu)["v"]


def _cta_of_points(P, grid, tile=128):
    """CTA of each point: tile t = point // 128 goes to CTA t % grid."""
    return (np.arange(P) // tile) % grid


def _chain_sum_err(terms, cta, grid, tiles_per_cta, axis_pts=0):
    """Error bound of a column sum over points (warp halving exchanges, one
    shared-memory atomic per warp and tile, one global atomic per CTA): a chain
    of at most 5 + 4 tiles_per_cta + grid additions, each with u times the
    running magnitude, bounded by the total magnitude."""
    n_chain = 5.0 + 4.0 * tiles_per_cta + grid
    return n_chain * U * np.abs(terms).sum(axis=axis_pts)


def _tc_grad_err(A, B, cta, grid, tiles_per_cta):
    """dW = A^T B accumulated on the tensor cores over each CTA's tiles (8 steps of
    K = 16 per 128-point tile), then added across CTAs by global atomics."""
    S = np.abs(A).T @ np.abs(B)
    err = 4.0 * (8.0 * tiles_per_cta + 1.0) * U_ACC * S
    T = np.zeros_like(S)
    for k in range(grid):
        sel = cta == k
        if sel.any():
            T += np.abs(A[sel].T @ B[sel])
    return err + grid * U * T


def gradient_bounds(p, lat, brick, x, target, grid, B=(16, 16, 16)):
    """Per-element bounds on the GPU's loss and gradients (W1, b1, W2, b2, w3,
    b3, lat) against ref.backward(..., bf=True) for a training step over these
    points run by `grid` CTAs of 128-point tiles."""
    P = len(brick)
    n_tiles = (P + 127) // 128
    tiles_per_cta = -(-n_tiles // grid)
    cta = _cta_of_points(P, grid)
    f = forward_terms(p, lat, brick, x, B)
    cache = {}
    ref.backward(p, lat, brick, x, target, bf=True, cache=cache)
    s = np.asarray(p["s"])[brick]
    W1q, W2q, w3q = f["W1q"], f["W2q"], f["w3q"]
    r = cache["v"] - target
    dr = f["v"] + U * np.abs(r)
    dy = cache["dy"]
    ddy = np.abs(s) * (2.0 / P) * dr + 3.0 * U * np.abs(dy)   # r s, times fl(2 / P)
    out = {}
    out["loss"] = (2.0 / P) * np.sum(np.abs(r) * dr) + 1e-12
    out["b3"] = np.array(ddy.sum() + _chain_sum_err(dy, cta, grid, tiles_per_cta))
    h2 = f["h2"]
    t3 = dy[:, None] * h2
    out["w3"] = (np.abs(dy)[:, None] * f["dh2"] + np.abs(h2) * ddy[:, None] + U * np.abs(t3)).sum(axis=0) \
        + _chain_sum_err(t3, cta, grid, tiles_per_cta)
    # layer-2 gradient before rounding: dy w3 silu'(z2), silu' from approximate
    # exp and division
    z2, sg2, sgg2 = f["z2"], f["sg2"], f["sgg2"]
    s2 = 1.0 / (1.0 + np.exp(-z2))
    e_sg2 = np.abs(1.0 + z2 * (1.0 - 2.0 * s2)) * (np.abs(z2) + 6.0) * 2.0 * U * s2 \
        + 4.0 * U * s2 * (1.0 + np.abs(z2) * (1.0 - s2))
    g2f = cache["g2f"]
    dg2f = np.abs(w3q)[None, :] * (np.abs(sg2) * ddy[:, None] + np.abs(dy)[:, None] *
                                   (np.abs(sgg2) * f["dz2"] + e_sg2)) + 3.0 * U * np.abs(g2f)
    out["b2"] = dg2f.sum(axis=0) + _chain_sum_err(g2f, cta, grid, tiles_per_cta)
    g2 = cache["g2"]
    dg2 = bf16_delta(g2f, dg2f)
    h1, dh1 = f["h1"], f["dh1"]
    out["W2"] = dg2.T @ np.abs(h1) + np.abs(g2).T @ dh1 + _tc_grad_err(g2, h1, cta, grid, tiles_per_cta)
    dH = cache["dh1"]
    ddH = dg2 @ np.abs(W2q) + _tc_err(np.abs(g2) @ np.abs(W2q), 64)
    z1, sg1, sgg1 = f["z1"], f["sg1"], f["sgg1"]
    s1 = 1.0 / (1.0 + np.exp(-z1))
    e_sg1 = np.abs(1.0 + z1 * (1.0 - 2.0 * s1)) * (np.abs(z1) + 6.0) * 2.0 * U * s1 \
        + 4.0 * U * s1 * (1.0 + np.abs(z1) * (1.0 - s1))
    g1f = cache["g1f"]
    dg1f = np.abs(sg1) * ddH + np.abs(dH) * (np.abs(sgg1) * f["dz1"] + e_sg1) + U * np.abs(g1f)
    out["b1"] = dg1f.sum(axis=0) + _chain_sum_err(g1f, cta, grid, tiles_per_cta)
    g1 = cache["g1"]
    dg1 = bf16_delta(g1f, dg1f)
    IN, dIN = f["IN"], f["dIN"]
    out["W1"] = dg1.T @ np.abs(IN) + np.abs(g1).T @ dIN + _tc_grad_err(g1, IN, cta, grid, tiles_per_cta)
    din = cache["din"]
    ddin = dg1 @ np.abs(W1q) + _tc_err(np.abs(g1) @ np.abs(W1q), 64)
    # latent gradients: w * din scattered to the 8 nodes by atomics in any order
    w, idx = f["w"], f["idx"]
    dw = 3.0 * U * w + 51.0 * U
    lat_err = np.zeros_like(lat, dtype=np.float64)
    lat_abs = np.zeros_like(lat, dtype=np.float64)
    lat_cnt = np.zeros(lat.shape[:4], dtype=np.float64)
    dz, ddz = din[:, :ref.LATENT], ddin[:, :ref.LATENT]
    for c in range(8):
        key = (brick, idx[:, c, 2], idx[:, c, 1], idx[:, c, 0])
        term = w[:, c:c + 1] * dz
        np.add.at(lat_err, key, np.abs(dz) * dw[:, c:c + 1] + w[:, c:c + 1] * ddz + U * np.abs(term))
        np.add.at(lat_abs, key, np.abs(term))
        np.add.at(lat_cnt, key, 1.0)
    out["lat"] = lat_err + lat_cnt[..., None] * U * lat_abs
    for k in out:
        out[k] = C * np.asarray(out[k]) + TINY
    out["flips"] = f["flips"] + int((dg2 > 0).sum() + (dg1 > 0).sum())
    out["ambiguous"] = f["ambiguous"] | big_flip(dg2, dg2f).any(axis=1) | big_flip(dg1, dg1f).any(axis=1)
    return out


def unambiguous_points(p, lat, brick, x, B=(16, 16, 16)):
    """Mask of points whose forward pass has no rounding decision that may go
    the other way by an amplifying step (big_flip).  These depend on the points
    alone, not on the batch; the backward pass's decisions (which scale with the
    batch's loss) stay in the bound, each touching only its own point's terms."""
    return ~forward_terms(p, lat, brick, x, B)["ambiguous"]
