"""Rank space on the GPU against the CPU oracle.

sky_rank_space's dense ranks and distinct counts are integer results and
must equal the oracle's bit for bit; its codes must equal the documented map
of those ranks.  A skyline computed with the rank images (SKY_IMAGES_RANKS)
must equal the oracle's in every index, partition and stage code: the images
only decide which pairs reach the engine's FP32 test.  The inputs include
value ranges where the FP16 images of the values are blunt (a large common
offset, magnitudes above the FP16 range, magnitudes near its bottom)."""
import numpy as np
import pytest

from paper_2411_14968_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2411_14968_gb300 import native
    c = native.Context(0)
    yield c
    c.close()


def _codes(ranks, distinct):
    """The code map that sky_rank_space documents: the rank itself for a
    column of at most RANK_CODES distinct values, else floor(rank x
    (RANK_CODES - 1) / (distinct - 1))."""
    from paper_2411_14968_gb300 import native
    rc = native.RANK_CODES
    r = ranks.astype(np.uint64)
    big = distinct.astype(np.uint64)[None, :]
    scaled = (r * (rc - 1)) // np.maximum(big - 1, 1)
    return np.where(big <= rc, r, scaled).astype(np.uint16)


def _cases():
    out = [datagen.anticorrelated(2001 + 13 * d, d, 60 + d) for d in range(1, 9)]
    q = np.round(datagen.independent(5000, 5, 61) * 8) / 8  # 9 values per column
    q[::7, 2] = -0.0  # -0.0 and +0.0 are one value
    out.append(q.astype(np.float32))
    out.append(np.array([[0.5, -3.0, 7.0]], np.float32))  # one point
    out.append(datagen.anticorrelated(40000, 3, 62))  # ~40,000 distinct per column: scaled codes
    return out


def test_rank_space_matches_oracle(ctx, oracle_mod, torch_cuda):
    torch = torch_cuda
    for x in _cases():
        want_r, want_d = oracle_mod.dense_ranks(x)
        want_c = _codes(want_r, want_d)
        tag = f"n={x.shape[0]} d={x.shape[1]}"
        r, dist, c = ctx.rank_space(x)  # host in, host out
        np.testing.assert_array_equal(dist, want_d, err_msg=tag)
        np.testing.assert_array_equal(r, want_r, err_msg=tag)
        np.testing.assert_array_equal(c, want_c, err_msg=tag)
        r, dist, c = ctx.rank_space(torch.from_numpy(x).cuda())  # device in, device out
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dist.cpu().numpy().astype(np.uint32), want_d, err_msg=tag)
        np.testing.assert_array_equal(r.cpu().numpy().astype(np.uint32), want_r, err_msg=tag)
        np.testing.assert_array_equal(c.cpu().numpy().view(np.uint16), want_c, err_msg=tag)
    big = _cases()[-1]
    _, d_big = oracle_mod.dense_ranks(big)
    assert (d_big > 31744).all()  # the scaled branch of the code map was exercised


def test_rank_space_edges(ctx, oracle_mod):
    from paper_2411_14968_gb300 import native
    r, dist, c = ctx.rank_space(np.zeros((0, 4), np.float32))
    assert r.shape == (0, 4) and c.shape == (0, 4)
    np.testing.assert_array_equal(dist, [0, 0, 0, 0])
    bad = datagen.independent(1000, 3, 63)
    bad[17, 1] = np.nan
    with pytest.raises(native.SkylineError) as e:
        ctx.rank_space(bad)
    assert e.value.status == native.SKY_EINVAL
    with pytest.raises(native.SkylineError) as e:
        ctx.skyline(bad, images="ranks")
    assert e.value.status == native.SKY_EINVAL
    # the context is still usable
    x = datagen.anticorrelated(3000, 4, 64)
    np.testing.assert_array_equal(ctx.skyline(x, images="ranks"), oracle_mod.skyline_indices(x))
    with pytest.raises(native.SkylineError) as e:
        ctx.skyline(x, params=native.make_params(images=7))
    assert e.value.status == native.SKY_EINVAL


TRANSFORMS = {
    "unit": lambda x: x,
    "offset": lambda x: x + np.float32(1024.0),          # FP16 spacing 1 there: ~2 images per column
    "large": lambda x: x * np.float32(2.0 ** 17),        # above 65504: clamped images
    "tiny": lambda x: x * np.float32(2.0 ** -20),        # FP16 subnormals: ~16 images per column
}

SCHEMES = [
    dict(scheme="none"),
    dict(scheme="random", p=16),
    dict(scheme="sliced", p=8),
    dict(scheme="grid", slices="g", normalize=True),
    dict(scheme="angular", slices="a", rep="sorted"),
    dict(scheme="sliced", p=8, merge="noseq"),
]


def _oracle_kw(kw, d):
    from oracle import oracle as O
    slices = kw.get("slices")
    if slices == "g":
        slices = [2] * d
    elif slices == "a":
        slices = [2] * (d - 1)
    return dict(scheme={"random": O.RANDOM, "grid": O.GRID, "angular": O.ANGULAR, "sliced": O.SLICED,
                        "none": O.NONE}[kw["scheme"]], p=kw.get("p", 1), slices=slices,
                normalize=kw.get("normalize", False), rep={"none": 0, "sorted": 1}[kw.get("rep", "none")],
                merge={"sequential": 0, "noseq": 1}[kw.get("merge", "sequential")])


@pytest.mark.parametrize("transform", list(TRANSFORMS))
@pytest.mark.parametrize("d", [2, 4, 6, 8])
def test_rank_images_skyline_matches_oracle(ctx, oracle_mod, transform, d):
    x = np.ascontiguousarray(TRANSFORMS[transform](datagen.anticorrelated(6000, d, 70 + d)), dtype=np.float32)
    for kw in SCHEMES:
        ok = _oracle_kw(kw, d)
        want = oracle_mod.partitioned(x, **ok)
        for images in ("ranks", "values"):
            args = dict(kw, slices=ok["slices"], images=images)
            idx, pid, stage = ctx.skyline(x, with_diag=True, **args)
            tag = f"{transform} d={d} {kw} images={images}"
            np.testing.assert_array_equal(idx, want["indices"], err_msg=tag)
            np.testing.assert_array_equal(pid, want["pid"], err_msg=tag + " pid")
            np.testing.assert_array_equal(stage, want["stage"], err_msg=tag + " stage")


def test_rank_images_in_a_batch(ctx, oracle_mod, torch_cuda):
    from paper_2411_14968_gb300 import native
    torch = torch_cuda
    xs = [datagen.anticorrelated(20000, 6, 80) + np.float32(1024.0), datagen.independent(5000, 3, 81),
          datagen.anticorrelated(50000, 5, 82) * np.float32(2.0 ** 17)]
    xs = [np.ascontiguousarray(x, dtype=np.float32) for x in xs]
    ps = [native.make_params(scheme="sliced", p=16, images="ranks"),
          native.make_params(scheme="none", images="values"),
          native.make_params(scheme="random", p=8, images="ranks")]
    got = ctx.skyline_batch([(torch.from_numpy(x).cuda(), p) for x, p in zip(xs, ps)])
    for x, g in zip(xs, got):
        np.testing.assert_array_equal(g.cpu().numpy().astype(np.uint32), oracle_mod.skyline_indices(x))


def test_rank_images_graph_serving_autotune(ctx, oracle_mod, torch_cuda):
    """Rank images through the other entry points: a captured batch replayed
    (also after its inputs are rewritten in place), the serving loop, and the
    autotuner, each checked against the oracle."""
    from paper_2411_14968_gb300 import native
    torch = torch_cuda
    O = oracle_mod
    off = np.float32(1024.0)
    x0 = [datagen.anticorrelated(30000, 5, 90) + off, datagen.independent(8000, 4, 91) * np.float32(2.0 ** 17)]
    x1 = [datagen.anticorrelated(30000, 5, 92) + off, datagen.independent(8000, 4, 93) * np.float32(2.0 ** 17)]
    x0 = [np.ascontiguousarray(x, dtype=np.float32) for x in x0]
    x1 = [np.ascontiguousarray(x, dtype=np.float32) for x in x1]
    ps = [native.make_params(scheme="sliced", p=8, rep="sorted", images="ranks"),
          native.make_params(scheme="grid", slices=[3] * 4, normalize=True, images="ranks")]
    ops = [dict(scheme=O.SLICED, p=8, rep=O.REP_SORTED), dict(scheme=O.GRID, slices=[3] * 4, normalize=True)]
    want0 = [O.partitioned(x, **kw)["indices"] for x, kw in zip(x0, ops)]
    want1 = [O.partitioned(x, **kw)["indices"] for x, kw in zip(x1, ops)]
    xt = [torch.from_numpy(x).cuda() for x in x0]
    g = ctx.capture(list(zip(xt, ps)))
    res, _ = g.run()
    for r, w in zip(res, want0):
        np.testing.assert_array_equal(r.cpu().numpy().astype(np.uint32), w)
    for t, x in zip(xt, x1):
        t.copy_(torch.from_numpy(x))
    res, _ = g.run()
    for r, w in zip(res, want1):
        np.testing.assert_array_equal(r.cpu().numpy().astype(np.uint32), w)
    g.close()
    # serving: rank-image and value-image queries in flight together
    ctx.serve_start(workers=2, max_batch=8)
    try:
        tickets = [(ctx.submit(x, p), w) for x, p, w in zip(x0 + x1, ps + ps, want0 + want1)]
        tickets.append((ctx.submit(x0[0], native.make_params(scheme="sliced", p=8, rep="sorted")), want0[0]))
        for t, w in tickets:
            got, _ = ctx.wait(t)
            np.testing.assert_array_equal(got, w)
    finally:
        ctx.serve_stop()
    # the autotuner keeps the method parameters (rank images included)
    tuned, ms = ctx.autotune(x0[0], params=ps[0], max_trials=6)
    assert ms > 0 and tuned.images == native.IMAGES["ranks"]
    np.testing.assert_array_equal(ctx.skyline(x0[0], params=tuned), want0[0])


def test_rank_images_extreme_values(ctx, oracle_mod):
    """Rank images of columns holding +-inf, -0.0 beside +0.0, subnormals,
    the largest finite values and long runs of one value: the same skyline,
    partitions and stage codes as the oracle's, and the same ranks."""
    rng = np.random.default_rng(95)
    x = datagen.anticorrelated(5000, 5, 95)
    special = np.array([np.inf, -np.inf, -0.0, 0.0, 1e-40, -1e-40, 3.4e38, -3.4e38, 7.0], np.float32)
    mask = rng.random(x.shape) < 0.05
    x[mask] = rng.choice(special, size=int(mask.sum()))
    x[:300, 1] = np.float32(0.25)  # a long run of one value
    x = np.ascontiguousarray(x, dtype=np.float32)
    want_r, want_d = oracle_mod.dense_ranks(x)
    r, dist, _ = ctx.rank_space(x)
    np.testing.assert_array_equal(dist, want_d)
    np.testing.assert_array_equal(r, want_r)
    for kw, okw in ((dict(scheme="none"), dict(scheme=oracle_mod.NONE)),
                    (dict(scheme="sliced", p=8, merge="noseq"), dict(scheme=oracle_mod.SLICED, p=8, merge=1)),
                    (dict(scheme="random", p=16, rep="sorted"), dict(scheme=oracle_mod.RANDOM, p=16, rep=1))):
        want = oracle_mod.partitioned(x, **okw)
        idx, pid, stage = ctx.skyline(x, images="ranks", with_diag=True, **kw)
        np.testing.assert_array_equal(idx, want["indices"], err_msg=str(kw))
        np.testing.assert_array_equal(pid, want["pid"], err_msg=str(kw))
        np.testing.assert_array_equal(stage, want["stage"], err_msg=str(kw))
