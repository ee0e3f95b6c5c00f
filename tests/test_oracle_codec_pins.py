"""Pins for the FP64 reference of the learned brick codec (oracle/codec.py):
finite differences for every gradient, closed forms of the forward pass, exact
interpolation of affine latent fields, known Fourier features and BF16 rounding."""
import numpy as np
import pytest

from oracle import codec


def _case(seed=3, n_bricks=3, P=64):
    rng = np.random.default_rng(seed)
    params, lat = codec.init_params(n_bricks, seed=seed, brick_mean=rng.normal(size=n_bricks),
                                    brick_scale=rng.uniform(0.5, 2.0, n_bricks))
    params["b1"] = rng.normal(0, 0.1, codec.HIDDEN)
    params["b2"] = rng.normal(0, 0.1, codec.HIDDEN)
    params["b3"] = np.array(0.2)
    brick = rng.integers(0, n_bricks, P)
    x = rng.uniform(0, 1, (P, 3))
    target = rng.normal(size=P)
    return params, lat, brick, x, target


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "w3", "b3", "lat"])
def test_gradients_match_finite_differences(name):
    params, lat, brick, x, target = _case()
    _, g = codec.backward(params, lat, brick, x, target, bf=False)
    rng = np.random.default_rng(11)
    base = lat if name == "lat" else params[name]
    flat = base.reshape(-1)
    gflat = g[name].reshape(-1)
    picks = rng.choice(flat.size, size=min(12, flat.size), replace=False)
    if name == "W1":
        picks = [k for k in picks if k % codec.K_IN < 28] or [0]   # the padded inputs are zero
    eps = 1e-6
    for k in picks:
        old = flat[k]
        flat[k] = old + eps
        lp = codec.backward(params, lat, brick, x, target, bf=False)[0]
        flat[k] = old - eps
        lm = codec.backward(params, lat, brick, x, target, bf=False)[0]
        flat[k] = old
        num = (lp - lm) / (2 * eps)
        assert abs(num - gflat[k]) <= 1e-6 * max(1.0, abs(num)), (name, k, num, gflat[k])


def test_silu_gradient():
    t = np.linspace(-8, 8, 101)
    num = (codec.silu(t + 1e-6) - codec.silu(t - 1e-6)) / 2e-6
    assert np.allclose(codec.silu_grad(t), num, atol=1e-8)
    assert codec.silu(0.0) == 0.0 and abs(codec.silu(50.0) - 50.0) < 1e-12


def test_fourier_features_known_values():
    f = codec.fourier(np.array([[0.0, 0.5, 1.0]]))[0]
    assert np.allclose(f[0:4], [0, 1, 0, 1])
    assert np.allclose(f[4:8], [1, 0, 0, -1], atol=1e-15)
    assert np.allclose(f[8:12], [0, -1, 0, 1], atol=1e-15)


def test_latent_interpolation_is_exact_on_nodes_and_affine_fields():
    rng = np.random.default_rng(2)
    lat = rng.normal(size=(1, 8, 8, 8, codec.LATENT))
    nodes = rng.integers(0, 8, (20, 3))
    z = codec.latent_interp(lat, np.zeros(20, dtype=np.int64), nodes / 7.0)
    assert np.allclose(z, lat[0, nodes[:, 2], nodes[:, 1], nodes[:, 0]])
    # affine latent field: node value a . (i, j, k) + c is reproduced everywhere
    a = rng.normal(size=(3, codec.LATENT))
    c = rng.normal(size=codec.LATENT)
    ii = np.arange(8)
    lat = (ii[None, None, :, None] * a[0] + ii[None, :, None, None] * a[1] + ii[:, None, None, None] * a[2]
           + c)[None]
    x = rng.uniform(0, 1, (50, 3))
    z = codec.latent_interp(lat, np.zeros(50, dtype=np.int64), x)
    assert np.allclose(z, (7 * x) @ a + c)


def test_forward_closed_form_with_zero_weights():
    params, lat, brick, x, _ = _case()
    params["W1"][:] = 0.0
    params["W2"][:] = 0.0
    v, _ = codec.forward(params, lat, brick, x, bf=False)
    y = codec.silu(params["b2"]) @ params["w3"] + params["b3"]
    assert np.allclose(v, y * params["s"][brick] + params["m"][brick])


def test_bf16_rounding():
    assert codec.bf16(1.0) == 1.0
    assert codec.bf16(1.0 + 2 ** -8) == 1.0                 # tie between 1 and 1 + 2^-7: even
    assert codec.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie: to the even mantissa
    assert codec.bf16(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    assert codec.bf16(-3.0) == -3.0 and codec.bf16(65280.0) == 65280.0


def test_bf16_mode_stays_close_to_the_exact_definition():
    params, lat, brick, x, target = _case()
    v1, _ = codec.forward(params, lat, brick, x, bf=True)
    v0, _ = codec.forward(params, lat, brick, x, bf=False)
    assert np.abs(v1 - v0).max() < 0.05 * (1 + np.abs(v0).max())
    assert np.abs(v1 - v0).max() > 0.0
