"""GPU checks of the learned brick codec's tensor-core path (tcgen05): products
through the shared-memory layouts and descriptors the codec kernels use, against
numpy in FP64 on the same BF16 values."""
import numpy as np
import pytest

from ooc_budget import budget_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("K,N", [(16, 16), (32, 64), (64, 32), (64, 64)])
def test_tensor_core_product(vr, a_mn, b_mn, K, N):
    rng = np.random.default_rng(K * 100 + N + 7 * a_mn + 13 * b_mn)
    A = vr.to_bf16_bits(rng.normal(size=(128, K)))
    B = vr.to_bf16_bits(rng.normal(size=(N, K)))
    D = vr.vr_codec_gemm_check(A, B, a_mn, b_mn)
    a = vr.bf16_bits_to_float(A).astype(np.float64)
    b = vr.bf16_bits_to_float(B).astype(np.float64)
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(D - ref) <= 1e-6 * scale + 1e-30)


# ------------------------------------------------------------------ the codec MLP

from oracle import codec as ref   # noqa: E402


def _setup(vr, n_bricks=3, brick=(16, 16, 16), seed=5):
    rng = np.random.default_rng(seed)
    params, lat = ref.init_params(n_bricks, seed=seed, brick_mean=rng.normal(size=n_bricks),
                                  brick_scale=rng.uniform(0.5, 2.0, n_bricks))
    params["b1"] = rng.normal(0, 0.2, 64)
    params["b2"] = rng.normal(0, 0.2, 64)
    params["b3"] = np.array(0.3)
    lat = rng.normal(0, 0.5, lat.shape)
    c = vr.Codec(n_bricks, brick)
    c.set_params(c.pack(params, lat), params["m"], params["s"])
    # the codec keeps FP32 parameters: compare against their FP32 values
    th, m, s = c.get_params()
    p = c.unpack(th.astype(np.float64))
    p["b3"] = p["b3"].reshape(())
    p["m"], p["s"] = m.astype(np.float64), s.astype(np.float64)
    return c, p, p["lat"], rng


def _points(rng, n, n_bricks, brick):
    """Seeded points; the positions are rounded to FP32 (what the kernel is given)."""
    bricks = rng.integers(0, n_bricks, n)
    u = rng.uniform(0, 1, (n, 3)) * np.array(brick)
    u[: n // 8] = np.round(u[: n // 8])          # lattice points too
    return bricks, u.astype(np.float32).astype(np.float64)


def test_codec_forward_matches_the_oracle(vr):
    """Every decoded value against the FP64 definition with the same BF16
    rounding points, within its own bound from the FP32/BF16 rounding model
    (tests/codec_bounds.py): FP32 accumulation and approximate SiLU everywhere,
    plus one BF16 step wherever the oracle's value lies within the GPU's error
    of a rounding boundary, propagated to the output."""
    from codec_bounds import forward_bound, forward_terms
    c, p, lat, rng = _setup(vr)
    bricks, u = _points(rng, 3000, 3, (16, 16, 16))
    got = c.forward(c.points(bricks, u)).astype(np.float64)
    x = u / 16.0
    want, _ = ref.forward(p, lat, bricks, x, bf=True)
    bound = forward_bound(p, lat, bricks, x)
    c.close()
    err = np.abs(got - want)
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, (bad[:5], err[bad[:5]], bound[bad[:5]])
    assert np.std(want) > 0.1
    # the bound is tight where no rounding decision can amplify an error
    clean = ~forward_terms(p, lat, bricks, x)["ambiguous"]
    assert clean.mean() > 0.4
    assert np.median(bound[clean] / (1.0 + np.abs(want[clean]))) < 1e-4


def test_codec_gradient_matches_the_oracle(vr):
    """Loss and every gradient element (W1, b1, W2, b2, w3, b3, each latent
    channel of each node) of a training step against the FP64 oracle, each
    within its own bound from the rounding model (tests/codec_bounds.py).  The
    batch keeps the points whose forward pass has no rounding decision that may
    go the other way by an amplifying step (the backward pass's decisions stay
    in the bound)."""
    import torch

    from codec_bounds import gradient_bounds, unambiguous_points
    c, p, lat, rng = _setup(vr)
    bricks, u = _points(rng, 6144, 3, (16, 16, 16))
    keep = unambiguous_points(p, lat, bricks, u / 16.0)
    bricks, u = bricks[keep], u[keep]
    assert len(bricks) > 2000
    targets = rng.normal(size=len(bricks)).astype(np.float32).astype(np.float64)
    loss, g = c.gradient(c.points(bricks, u), targets)
    x = u / 16.0
    want_loss, want = ref.backward(p, lat, bricks, x, targets, bf=True)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_tiles = (len(bricks) + 127) // 128
    bounds = gradient_bounds(p, lat, bricks, x, targets, grid=min(n_tiles, 2 * sms))
    c.close()
    got = c.unpack(g.astype(np.float64))
    assert abs(loss - want_loss) <= bounds["loss"], (loss, want_loss, bounds["loss"])
    for name in ("W1", "b1", "W2", "b2", "w3", "b3", "lat"):
        a, b, e = got[name], np.asarray(want[name]), bounds[name]
        if name == "W1":
            a, b, e = a[:, :28], b[:, :28], e[:, :28]
        a, b, e = a.reshape(-1), b.reshape(-1), e.reshape(-1)
        bad = np.flatnonzero(np.abs(a - b) > e)
        assert bad.size == 0, (name, bad[:5], a[bad[:5]], b[bad[:5]], e[bad[:5]])
        # the largest element of each block is pinned to well under 1%
        k = int(np.argmax(np.abs(b)))
        assert e[k] < 1e-2 * abs(b[k]), (name, e[k], b[k])
    assert np.abs(got["W1"][:, 28:]).max() == 0.0   # the padded inputs are zero


def test_codec_decodes_brick_blocks(vr):
    """Brick blocks decoded for rendering (SiLU through the hardware tanh) against
    the FP64 oracle at every voxel of the block, within the rounding-model bound
    with the tanh's error, and against the point queries within the same bound."""
    import torch

    from codec_bounds import forward_bound
    brick = (8, 12, 10)
    c, p, lat, rng = _setup(vr, n_bricks=4, brick=brick)
    ids = torch.tensor([2, 0], dtype=torch.int32, device="cuda")
    V = 9 * 13 * 11
    out = torch.zeros(2 * V, dtype=torch.float32, device="cuda")
    c.decode_bricks(ids, out)
    torch.cuda.synchronize()
    q = np.arange(V)
    u = np.stack([q % 9, (q // 9) % 13, q // (9 * 13)], axis=1).astype(np.float64)
    x = u / np.array(brick, dtype=np.float64)
    for k, b in enumerate([2, 0]):
        got = out[k * V:(k + 1) * V].cpu().numpy().astype(np.float64)
        bricks = np.full(V, b)
        want, _ = ref.forward(p, lat, bricks, x, bf=True)
        bound = forward_bound(p, lat, bricks, x, brick, fast_silu=True)
        bad = np.flatnonzero(np.abs(got - want) > bound)
        assert bad.size == 0, (b, bad[:5], got[bad[:5]], want[bad[:5]], bound[bad[:5]])
        direct = c.forward(c.points(bricks, u)).astype(np.float64)
        assert np.all(np.abs(got - direct) <= bound + forward_bound(p, lat, bricks, x, brick))
        assert np.median(np.abs(got - want) / (1.0 + np.abs(want))) < 1e-3
    c.close()


def test_codec_training_fits_a_cube(vr):
    """Adam on voxels of a smooth synthetic cube (Gaussian sources, no noise)
    lowers the loss by 10x."""
    import torch

    import synth
    cube = np.zeros((33, 33, 33), np.float32)
    synth.add_sources(cube, synth.line_sources(np.random.default_rng(21), 6, (33, 33, 33), (2.0, 8.0),
                                               (4.0, 10.0), (4.0, 12.0)))
    brick = (16, 16, 16)
    nb = 2 * 2 * 2
    dev = torch.from_numpy(cube).cuda()
    p, lat = ref.init_params(nb, seed=3)
    with vr.Codec(nb, brick) as c:
        c.set_params(c.pack(p, lat), np.zeros(nb), np.ones(nb))
        c.fit_stats(dev)
        th, m, s = c.get_params()
        c.set_params(th, m, s)
        rng = np.random.default_rng(0)
        bricks, u = _points(rng, 4096, nb, brick)
        bi = np.asarray(bricks)
        gx = np.minimum((bi % 2) * 16 + np.round(u[:, 0]).astype(int), 32)
        gy = np.minimum(((bi // 2) % 2) * 16 + np.round(u[:, 1]).astype(int), 32)
        gz = np.minimum((bi // 4) * 16 + np.round(u[:, 2]).astype(int), 32)
        u = np.stack([gx - (bi % 2) * 16, gy - ((bi // 2) % 2) * 16, gz - (bi // 4) * 16], axis=1)
        target = cube[gz, gy, gx]
        before = np.mean((c.forward(c.points(bricks, u)) - target) ** 2)
        c.train(dev, steps=300, batch=8192, lr=3e-3, seed=9)
        after = np.mean((c.forward(c.points(bricks, u)) - target) ** 2)
    assert after < 0.1 * before, (before, after)


def test_codec_decodes_into_slots_and_renders(vr):
    """Learned residency: bricks decoded into cache slots render the same image as
    the decoded cube rendered in core (the codec's cube, materialised by decoding
    every brick), and the image is close to the original cube's after training."""
    import torch

    import synth
    shape, brick = (33, 33, 33), (16, 16, 16)
    cube = np.zeros((33, 33, 33), np.float32)
    synth.add_sources(cube, synth.line_sources(np.random.default_rng(21), 6, shape, (2.0, 8.0),
                                               (4.0, 10.0), (4.0, 12.0)))
    tf = synth.make_tf([0.0, 0.02, 0.05, 0.1, 0.15, 0.2, 0.3, 0.4], lo=0.0, hi=8.0)
    dev = torch.from_numpy(cube).cuda()
    nb = 8
    p, lat = ref.init_params(nb, seed=3)
    with vr.Codec(nb, brick) as c:
        c.set_params(c.pack(p, lat), np.zeros(nb), np.ones(nb))
        c.fit_stats(dev)
        th, m, s = c.get_params()
        c.set_params(th, m, s)
        c.train(dev, steps=400, batch=8192, lr=3e-3, seed=9)
        # the decoded cube: every brick's block, the owned voxels put in place
        ids = torch.arange(nb, dtype=torch.int32, device="cuda")
        blocks = torch.zeros(nb * 17 ** 3, dtype=torch.float32, device="cuda")
        c.decode_bricks(ids, blocks)
        torch.cuda.synchronize()
        blk = blocks.cpu().numpy().reshape(nb, 17, 17, 17)
        decoded = np.zeros_like(cube)
        for b in range(nb):
            bx, by, bz = b % 2, (b // 2) % 2, b // 4
            decoded[bz * 16:bz * 16 + 17, by * 16:by * 16 + 17, bx * 16:bx * 16 + 17] = blk[b]
        # owners win at shared faces: write each brick's own voxels last-in-order of ownership
        for b in range(nb):
            bx, by, bz = b % 2, (b // 2) % 2, b // 4
            z1 = 17 if bz == 1 else 16
            y1 = 17 if by == 1 else 16
            x1 = 17 if bx == 1 else 16
            decoded[bz * 16:bz * 16 + z1, by * 16:by * 16 + y1, bx * 16:bx * 16 + x1] = blk[b, :z1, :y1, :x1]
        cam = synth.pose(shape, 0.7, 0.3, 96, 80)
        for budget in (0, 3):
            with vr.VolumeRenderer(0) as r:
                r.load_cube_codec(c, shape)
                if budget:
                    r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget * 17 ** 3 * 4)   # 3 blocks: a 2-slot cache
                r.brick(*brick)
                r.set_transfer_function(tf)
                r.set_camera(cam)
                learned = r.render().cpu().numpy()
                st = r.stats()
            assert st["device_errors"] == 0
            assert st["bricks_uploaded"] > 0
            ref_img = _render_incore(vr, torch, decoded, tf, cam, brick)
            # the in-core march reads each apron voxel from its owner, the slot
            # march from the reading brick's own decode: they agree where the two
            # decodes of a face voxel agree
            assert np.abs(learned - ref_img).max() < 0.05
        plain = _render_incore(vr, torch, cube, tf, cam, brick)
        mse = np.mean((learned.astype(np.float64) - plain) ** 2)
        psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
        assert psnr > 30.0, psnr


def _render_incore(vr, torch, cube, tf, cam, brick):
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(np.ascontiguousarray(cube, dtype=np.float32)).cuda())
        r.brick(*brick)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        r.set_option(vr.VR_OPT_KERNEL, vr.VR_KERNEL_DIRECT)
        return r.render().cpu().numpy()


# ------------------------------------------------ per-brick fallback to plain voxels

def _fallback_case(vr, torch):
    """A ragged cube (3 x 2 x 2 bricks of 16, the last ones partial) and a codec
    trained briefly on it, so that the bricks' decode errors spread."""
    import synth
    shape, brick = (40, 33, 29), (16, 16, 16)
    cube = np.zeros(shape[::-1], np.float32)
    synth.add_sources(cube, synth.line_sources(np.random.default_rng(33), 9, shape, (2.0, 8.0),
                                               (3.0, 8.0), (3.0, 10.0)))
    cube += np.random.default_rng(34).normal(0, 0.05, cube.shape).astype(np.float32)
    nb = 3 * 2 * 2
    p, lat = ref.init_params(nb, seed=4)
    c = vr.Codec(nb, brick)
    c.set_params(c.pack(p, lat), np.zeros(nb), np.ones(nb))
    dev = torch.from_numpy(cube).cuda()
    c.fit_stats(dev)
    th, m, s = c.get_params()
    c.set_params(th, m, s)
    c.train(dev, steps=150, batch=4096, lr=3e-3, seed=2)
    tf = synth.make_tf([0.0, 0.02, 0.05, 0.1, 0.15, 0.2, 0.3, 0.4], lo=0.0, hi=8.0)
    cam = synth.pose(shape, 0.9, 0.35, 72, 56)
    return cube, shape, brick, c, tf, cam


def _ctx(vr, shape, brick, tf, cam, codec=None, cube=None, fallback=None, budget=0, floor=-3.4e38, march=1):
    """A plain or learned context on the texture march (march=1: three layered
    copies per slot plus a staging area) or on the direct march (march=0: a block
    per slot), with a cache of `budget` slots (0: every brick)."""
    r = vr.VolumeRenderer(0)
    if codec is not None:
        r.load_cube_codec(codec, shape)
        if fallback is not None:
            r.set_codec_fallback(cube, fallback, floor)
    else:
        r.load_cube_host(cube)
    r.set_option(vr.VR_OPT_OOC_MARCH, march)
    if budget:
        r.set_option(vr.VR_OPT_DEVICE_BUDGET, budget_for(budget, brick, march))
    r.set_option(vr.VR_OPT_SKIP_EMPTY, 0)   # codec and plain ranges may differ
    r.brick(*brick)
    r.set_transfer_function(tf)
    r.set_camera(cam)
    return r


def test_fallback_errors_are_the_decoded_blocks_errors(vr):
    """The scan's per-brick error is max |max(d, f) - max(v, f)| over the brick's
    block inside the cube, d from vr_codec_decode_bricks, v the plain cube."""
    import torch
    cube, shape, brick, c, tf, cam = _fallback_case(vr, torch)
    nb = 12
    ids = torch.arange(nb, dtype=torch.int32, device="cuda")
    blocks = torch.zeros(nb * 17 ** 3, dtype=torch.float32, device="cuda")
    c.decode_bricks(ids, blocks)
    torch.cuda.synchronize()
    blk = blocks.cpu().numpy().reshape(nb, 17, 17, 17)
    for floor in (np.float32(-3.4e38), np.float32(0.7)):
        want = np.zeros(nb, np.float32)
        for b in range(nb):
            ix, iy, iz = b % 3, (b // 3) % 2, b // 6
            x0, y0, z0 = 16 * ix, 16 * iy, 16 * iz
            v = cube[z0:z0 + 17, y0:y0 + 17, x0:x0 + 17]
            d = blk[b, :v.shape[0], :v.shape[1], :v.shape[2]]
            want[b] = np.abs(np.maximum(d, floor) - np.maximum(v, floor)).max()
        with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=float(np.median(want)),
                  floor=float(floor)) as r:
            got, n_plain = r.codec_brick_errors()
        assert np.array_equal(got, want), (got, want)
        assert n_plain == int(np.sum(want > np.float32(np.median(want))))
        assert want.max() > 0
    c.close()


def test_fallback_extremes_equal_plain_streaming_and_pure_decoding(vr):
    """bound < 0: every brick is copied from its plain block, the image is the
    out-of-core plain render's bit for bit; bound = inf: the pure learned render."""
    import torch
    cube, shape, brick, c, tf, cam = _fallback_case(vr, torch)
    for budget in (0, 3):
        with _ctx(vr, shape, brick, tf, cam, cube=cube, budget=budget) as r:
            plain = r.render().cpu().numpy()
        with _ctx(vr, shape, brick, tf, cam, codec=c, budget=budget) as r:
            learned = r.render().cpu().numpy()
        with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=-1.0, budget=budget) as r:
            every = r.render().cpu().numpy()
            assert r.codec_brick_errors()[1] == 12
            st = r.stats()
        assert st["device_errors"] == 0 and st["bricks_uploaded"] > 0
        with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=float("inf"), budget=budget) as r:
            none = r.render().cpu().numpy()
            assert r.codec_brick_errors()[1] == 0
        assert np.array_equal(every, plain)
        assert np.array_equal(none, learned)
        assert not np.array_equal(plain, learned)
        assert plain[..., 3].max() > 0.3
    c.close()


def test_fallback_routes_each_brick(vr):
    """With the bound at the median error, each brick alone (a one-brick region)
    renders as the plain render if its error exceeds the bound and as the learned
    render otherwise; the whole frame is the same with every brick resident and
    streamed through a 3-slot cache, and closer to the plain image than the pure
    learned one."""
    import torch
    cube, shape, brick, c, tf, cam = _fallback_case(vr, torch)
    with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=float("inf")) as r:
        err, _ = r.codec_brick_errors()
    bound = float(np.median(err))
    flagged = err > np.float32(bound)
    assert 0 < flagged.sum() < 12
    mixed = _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=bound)
    plain = _ctx(vr, shape, brick, tf, cam, cube=cube)
    learned = _ctx(vr, shape, brick, tf, cam, codec=c)
    seen = 0
    for b in range(12):
        ix, iy, iz = b % 3, (b // 3) % 2, b // 6
        lo, hi = (ix, iy, iz), (ix + 1, iy + 1, iz + 1)
        imgs = []
        for r in (mixed, plain, learned):
            r.set_region(lo, hi)
            imgs.append(r.render().cpu().numpy())
        want = imgs[1] if flagged[b] else imgs[2]
        assert np.array_equal(imgs[0], want), b
        seen += int(imgs[0][..., 3].max() > 0)
    assert seen >= 6
    full = []
    for r in (mixed, plain, learned):
        r.set_region((0, 0, 0), (3, 2, 2))
        full.append(r.render().cpu().numpy())
    for r in (mixed, plain, learned):
        r.close()
    with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=bound, budget=3) as r:
        streamed = r.render().cpu().numpy()
        assert r.stats()["bricks_uploaded"] > 0
    assert np.array_equal(streamed, full[0])
    mse = lambda a: float(np.mean((a.astype(np.float64) - full[1]) ** 2))
    assert mse(full[0]) < mse(full[2])
    c.close()


def test_fallback_errors(vr):
    import torch
    cube = np.zeros((20, 20, 20), np.float32)
    with vr.VolumeRenderer(0) as r:
        r.load_cube(torch.from_numpy(cube).cuda())
        with pytest.raises(vr.VRError, match="VR_ESTATE"):
            r.set_codec_fallback(cube, 1.0)
    with vr.Codec(8, (10, 10, 10)) as c, vr.VolumeRenderer(0) as r:
        r.load_cube_codec(c, (20, 20, 20))
        with pytest.raises(vr.VRError, match="VR_EINVAL"):
            r.set_codec_fallback(cube, float("nan"))
        r.brick(10, 10, 10)
        with pytest.raises(vr.VRError, match="VR_ESTATE"):
            r.codec_brick_errors()     # no fallback was set


def test_what_training_and_the_fallback_gain(vr):
    """What the learned form gains over the method without it, on a 64³ cube of
    32³ bricks: training raises the PSNR against the plain render by 10 dB or more
    over the untrained network, while the device holds 16 KiB of latents per
    brick instead of its 140 KiB block; the fallback at the median brick error
    raises the PSNR further and pins plain blocks for only part of the bricks."""
    import torch

    import synth
    shape, brick = (64, 64, 64), (32, 32, 32)
    cube = np.zeros((64, 64, 64), np.float32)
    synth.add_sources(cube, synth.line_sources(np.random.default_rng(41), 10, shape, (2.0, 8.0),
                                               (4.0, 10.0), (4.0, 12.0)))
    tf = synth.make_tf([0.0, 0.02, 0.05, 0.1, 0.15, 0.2, 0.3, 0.4], lo=0.0, hi=8.0)
    cam = synth.pose(shape, 0.6, 0.3, 96, 96)
    nb = 8
    dev = torch.from_numpy(cube).cuda()

    def render(c, fallback=None):
        with _ctx(vr, shape, brick, tf, cam, codec=c, cube=cube, fallback=fallback) as r:
            img = r.render().cpu().numpy().astype(np.float64)
            n_plain = r.codec_brick_errors()[1] if fallback is not None else 0
            errs = r.codec_brick_errors()[0] if fallback is not None else None
        return img, n_plain, errs

    with _ctx(vr, shape, brick, tf, cam, cube=cube) as r:
        plain = r.render().cpu().numpy().astype(np.float64)
    psnr = lambda img: 10 * np.log10(1.0 / max(float(np.mean((img - plain) ** 2)), 1e-30))
    p, lat = ref.init_params(nb, seed=6)
    with vr.Codec(nb, brick) as c:
        c.set_params(c.pack(p, lat), np.zeros(nb), np.ones(nb))
        c.fit_stats(dev)
        th, m, s = c.get_params()
        c.set_params(th, m, s)
        untrained = psnr(render(c)[0])
        c.train(dev, steps=400, batch=8192, lr=3e-3, seed=3)
        trained = psnr(render(c)[0])
        _, _, errs = render(c, float("inf"))
        bound = float(np.median(errs))
        mixed_img, n_plain, _ = render(c, bound)
        mixed = psnr(mixed_img)
    latent_bytes, block_bytes = 8 ** 3 * 16 * 2, 33 ** 3 * 4
    assert block_bytes > 8 * latent_bytes
    assert trained >= untrained + 10.0, (untrained, trained)
    assert 0 < n_plain < nb
    assert mixed > trained, (trained, mixed)


# ------------------------------------------------ slab-by-slab fitting and training

def _slab_case(vr, n_codecs=2):
    """A ragged cube of 3 x 2 x 3 bricks of 16 (layers bz = 0, 1, 2, the last ones
    partial) and codecs with the same initial parameters."""
    import torch

    import synth
    shape, brick = (40, 33, 45), (16, 16, 16)
    cube = np.zeros(shape[::-1], np.float32)
    synth.add_sources(cube, synth.line_sources(np.random.default_rng(41), 12, shape, (2.0, 8.0),
                                               (3.0, 8.0), (3.0, 10.0)))
    cube += np.random.default_rng(42).normal(0, 0.05, cube.shape).astype(np.float32)
    nb = 3 * 2 * 3
    p, lat = ref.init_params(nb, seed=6)
    codecs = []
    for _ in range(n_codecs):
        c = vr.Codec(nb, brick)
        c.set_params(c.pack(p, lat), np.zeros(nb), np.ones(nb))
        codecs.append(c)
    return torch.from_numpy(cube).cuda(), shape, brick, nb, codecs


def _slab(dev, bz0, bz1, bz=16):
    return dev[bz0 * bz: min(bz1 * bz, dev.shape[0] - 1) + 1].contiguous()


@pytest.mark.parametrize("floor", [-3.4e38, 0.5])
def test_slab_fitting_and_training_equal_the_whole_cube(vr, floor):
    """fit_stats slab by slab gives every brick's offset, scale and range of the
    whole-cube fit bit for bit.  Training over all layers at once (slab = the
    cube) draws the same points as vr_codec_train: the two agree to within the
    run-to-run spread of vr_codec_train itself (its gradient sums use atomics, so
    two runs differ in rounding), far closer than a run with another seed."""
    dev, shape, brick, nb, (a, a2, b, c) = _slab_case(vr, 4)
    for x in (a, a2):
        x.fit_stats(dev, floor)
    for x in (b, c):
        for bz0, bz1 in ((0, 1), (1, 3)):
            x.fit_stats_slab(_slab(dev, bz0, bz1), shape, bz0, bz1, floor)
    ta, ma, sa = a.get_params()
    tb, mb, sb = b.get_params()
    assert np.array_equal(a.minmax(), b.minmax())
    assert np.array_equal(ma, mb) and np.array_equal(sa, sb)
    la = a.train(dev, steps=25, batch=4096, lr=3e-3, seed=3)
    a2.train(dev, steps=25, batch=4096, lr=3e-3, seed=3)
    lb = b.train_slab(dev, shape, 0, 3, steps=25, batch=4096, lr=3e-3, seed=3)
    c.train_slab(dev, shape, 0, 3, steps=25, batch=4096, lr=3e-3, seed=4)
    ta, ta2, tb, tc = (x.get_params()[0].astype(np.float64) for x in (a, a2, b, c))
    spread = max(3 * np.mean(np.abs(ta - ta2)), 1e-5)
    assert abs(la - lb) <= 1e-4 * abs(la)
    assert np.mean(np.abs(ta - tb)) <= spread
    assert np.mean(np.abs(ta - tc)) > 10 * spread
    for x in (a, a2, b, c):
        x.close()


def test_slab_training_touches_only_its_latents(vr):
    """Training slab [1, 2): the other layers' latents stay bit for bit; with
    mlp_lr = 0 the shared network stays too, and the slab's loss falls as its
    latents (reset to noise) are fitted again to the trained decoder."""
    import torch
    dev, shape, brick, nb, (a, b) = _slab_case(vr)
    for bz0, bz1 in ((0, 1), (1, 2), (2, 3)):
        a.fit_stats_slab(_slab(dev, bz0, bz1), shape, bz0, bz1)
    a.train_slab(dev, shape, 0, 3, steps=300, batch=8192, lr=3e-3, seed=2)     # decoder and latents
    th, m, s = a.get_params()
    n_mlp = a.n_params - nb * 8 ** 3 * 16
    lat_of = lambda th, b0, b1: th[n_mlp + b0 * 8192: n_mlp + b1 * 8192]   # noqa: E731
    lat_of(th, 6, 12)[:] = np.random.default_rng(8).normal(0, 0.1, 6 * 8192)
    a.set_params(th, m, s)
    th0 = a.get_params()[0]
    slab = _slab(dev, 1, 2)
    first = a.train_slab(slab, shape, 1, 2, steps=1, batch=8192, lr=3e-3, mlp_lr=0.0, seed=4)
    last = a.train_slab(slab, shape, 1, 2, steps=200, batch=8192, lr=3e-3, mlp_lr=0.0, seed=5)
    th1 = a.get_params()[0]
    assert np.array_equal(th1[:n_mlp], th0[:n_mlp])
    assert np.array_equal(lat_of(th1, 0, 6), lat_of(th0, 0, 6))
    assert np.array_equal(lat_of(th1, 12, 18), lat_of(th0, 12, 18))
    assert not np.array_equal(lat_of(th1, 6, 12), lat_of(th0, 6, 12))
    assert last < 0.7 * first, (first, last)
    # with the network's rate on, the network moves and the other latents still stay
    a.train_slab(slab, shape, 1, 2, steps=5, batch=4096, lr=3e-3, mlp_lr=1e-3, seed=6)
    th2 = a.get_params()[0]
    assert not np.array_equal(th2[:n_mlp], th1[:n_mlp])
    assert np.array_equal(lat_of(th2, 0, 6), lat_of(th0, 0, 6))
    # decoding reflects the slab's latents only: bricks of layer 0 decode as before
    ids = torch.arange(6, dtype=torch.int32, device="cuda")
    out = torch.empty(6 * 17 ** 3, device="cuda")
    b.set_params(*a.get_params())
    with pytest.raises(vr.VRError):
        b.train_slab(dev[32:].contiguous(), shape, 2, 4, steps=1, batch=16, lr=1e-3)   # layers beyond the cube
    with pytest.raises(ValueError):
        b.train_slab(_slab(dev, 0, 2), shape, 1, 2, steps=1, batch=16, lr=1e-3)   # wrong plane count
    b.decode_bricks(ids, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    a.close()
    b.close()
