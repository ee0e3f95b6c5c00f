"""CPU checks of the per-element comparison used by the codec's GPU parity tests
(tests/codec_bounds.py): the bounds admit FP32 roundings of the oracle's own
values, and reject a single element moved by 1% or a dropped BF16 rounding
point.  No GPU: the "GPU values" here are made from the oracle."""
import numpy as np
import pytest

from codec_bounds import forward_bound, forward_terms, gradient_bounds, unambiguous_points
from oracle import codec as ref

BLOCKS = ("W1", "b1", "W2", "b2", "w3", "b3", "lat")


def _case(seed=5, n_bricks=3, P=3000):
    rng = np.random.default_rng(seed)
    params, lat = ref.init_params(n_bricks, seed=seed, brick_mean=rng.normal(size=n_bricks),
                                  brick_scale=rng.uniform(0.5, 2.0, n_bricks))
    params["b1"] = rng.normal(0, 0.2, 64)
    params["b2"] = rng.normal(0, 0.2, 64)
    params["b3"] = np.array(0.3)
    lat = rng.normal(0, 0.5, lat.shape)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)   # noqa: E731
    params = {k: f32(v) for k, v in params.items()}
    bricks = rng.integers(0, n_bricks, P)
    u = f32(rng.uniform(0, 1, (P, 3)) * 16.0)
    return params, f32(lat), bricks, u / 16.0, rng


def _violations(got, want, bound):
    return int(np.sum(np.abs(np.asarray(got) - np.asarray(want)) > np.asarray(bound)))


def test_forward_bound_admits_fp32_and_rejects_a_one_percent_change():
    p, lat, bricks, x, _ = _case()
    want, _ = ref.forward(p, lat, bricks, x, bf=True)
    bound = forward_bound(p, lat, bricks, x)
    assert _violations(np.float32(want), want, bound) == 0
    clean = np.flatnonzero(~forward_terms(p, lat, bricks, x)["ambiguous"])
    assert clean.size > 1000
    for k in clean[:50]:
        got = np.float32(want).astype(np.float64)
        got[k] *= 1.01
        assert _violations(got, want, bound) == 1


def test_forward_bound_rejects_a_dropped_rounding_point():
    """The latents enter the interpolation as BF16 values; an implementation that
    interpolated the FP32 master latents instead is caught at many points."""
    p, lat, bricks, x, _ = _case()
    want, _ = ref.forward(p, lat, bricks, x, bf=True)
    bound = forward_bound(p, lat, bricks, x)
    lat_f32 = lat.copy()
    mutant = dict(p)
    # the mutant forward: BF16 rounding of the latents skipped (rows still rounded)
    IN = ref.bf16(np.concatenate([ref.latent_interp(lat_f32, bricks, x), ref.fourier(x),
                                  np.zeros((len(bricks), ref.K_IN - ref.LATENT - 12))], axis=1))
    q = ref.bf16
    h1 = q(ref.silu(IN @ q(mutant["W1"]).T + mutant["b1"]))
    h2 = ref.silu(h1 @ q(mutant["W2"]).T + mutant["b2"])
    got = (h2 @ q(mutant["w3"]) + mutant["b3"]) * mutant["s"][bricks] + mutant["m"][bricks]
    assert _violations(got, want, bound) > 0.2 * len(bricks)


@pytest.fixture(scope="module")
def grad_case():
    p, lat, bricks, x, rng = _case(P=4096)
    keep = unambiguous_points(p, lat, bricks, x)
    bricks, x = bricks[keep], x[keep]
    targets = rng.normal(size=len(bricks)).astype(np.float32).astype(np.float64)
    loss, want = ref.backward(p, lat, bricks, x, targets, bf=True)
    bounds = gradient_bounds(p, lat, bricks, x, targets, grid=(len(bricks) + 127) // 128)
    return loss, want, bounds


def test_gradient_bounds_admit_fp32_roundings(grad_case):
    loss, want, bounds = grad_case
    assert abs(np.float32(loss) - loss) <= bounds["loss"]
    for name in BLOCKS:
        w = np.asarray(want[name])
        assert _violations(w.astype(np.float32), w, bounds[name]) == 0, name


@pytest.mark.parametrize("name", BLOCKS)
def test_gradient_bounds_reject_one_element_moved_by_one_percent(grad_case, name):
    """The largest element of the block moved by 1% fails the comparison, and so
    does a typical element for all but the cancellation-heavy blocks."""
    _, want, bounds = grad_case
    w = np.asarray(want[name], dtype=np.float64).reshape(-1)
    e = np.asarray(bounds[name]).reshape(-1)
    if name == "W1":
        w = np.asarray(want[name])[:, :28].reshape(-1)
        e = np.asarray(bounds[name])[:, :28].reshape(-1)
    k = int(np.argmax(np.abs(w)))
    got = w.astype(np.float32).astype(np.float64)
    got[k] *= 1.01
    assert _violations(got, w, e) == 1
    # share of elements whose bound is under 1% of their value
    nz = np.abs(w) > 0
    share = np.mean(e[nz] < 1e-2 * np.abs(w[nz]))
    assert share > {"W1": 0.25, "lat": 0.5}.get(name, 0.9), (name, share)
