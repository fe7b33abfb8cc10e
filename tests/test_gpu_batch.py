"""Batches of independent queries (sky_skyline_batch): every query's result
must equal the oracle's for that query alone, whatever else shares its
engine launches."""
import numpy as np
import pytest

from paper_2411_14968_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_14968_gb300 import native
    c = native.Context(0)
    yield c
    c.close()


def _mix():
    from oracle import oracle as O
    # (points, binding keyword arguments, oracle keyword arguments)
    return [
        (datagen.anticorrelated(20000, 6, 31), dict(scheme="sliced", p=8, rep="sorted"),
         dict(scheme=O.SLICED, p=8, rep=1)),
        (datagen.independent(5000, 3, 32), dict(scheme="grid", slices=[3, 3, 3]),
         dict(scheme=O.GRID, slices=[3, 3, 3])),
        (datagen.correlated(8000, 8, 33), dict(scheme="angular", slices=[2] * 7),
         dict(scheme=O.ANGULAR, slices=[2] * 7)),
        (datagen.make("skewed", 3000, 5, 34), dict(scheme="random", p=4, seed=5, merge="noseq"),
         dict(scheme=O.RANDOM, p=4, seed=5, merge=1)),
        (datagen.independent(1, 4, 35), dict(), dict()),
        (np.zeros((0, 3), np.float32), dict(scheme="sliced", p=3), dict(scheme=O.SLICED, p=3)),
        (datagen.anticorrelated(12000, 4, 36), dict(scheme="sliced", p=5, exec="plain"),
         dict(scheme=O.SLICED, p=5)),
        (datagen.anticorrelated(30000, 5, 37), dict(), dict()),
    ]


def test_batch_matches_oracle(ctx, oracle_mod):
    import torch
    from paper_2411_14968_gb300 import native
    mix = _mix()
    queries = []
    for i, (x, kw, _) in enumerate(mix):
        pts = torch.from_numpy(x).cuda() if i % 2 else x  # host and device inputs mixed
        queries.append((pts, native.make_params(**kw)))
    got = ctx.skyline_batch(queries)
    torch.cuda.synchronize()
    for (x, kw, okw), g in zip(mix, got):
        if hasattr(g, "cpu"):
            g = g.cpu().numpy()
        want = oracle_mod.partitioned(x, **okw)["indices"] if x.shape[0] else np.zeros(0, np.uint32)
        np.testing.assert_array_equal(np.asarray(g).astype(np.uint32), want, err_msg=str(kw))


def test_batch_equals_single_calls(ctx):
    from paper_2411_14968_gb300 import native
    xs = [datagen.anticorrelated(n, d, 40 + n % 7) for n, d in ((50000, 6), (7000, 3), (90000, 8), (3000, 5))]
    params = [native.make_params(scheme="sliced", p=16), native.make_params(scheme="angular", slices=[3, 2]),
              native.make_params(scheme="random", p=32, seed=3, rep="sorted"), native.make_params()]
    single = [ctx.skyline(x, params=p) for x, p in zip(xs, params)]
    for _ in range(2):  # the second batch reuses the workspace the first left behind
        got = ctx.skyline_batch(list(zip(xs, params)))
        for s, g in zip(single, got):
            np.testing.assert_array_equal(g, s)


def test_batch_rejects_invalid_query(ctx):
    from paper_2411_14968_gb300 import native
    good = datagen.independent(100, 3, 1)
    bad = good.copy()
    bad[5, 0] = np.nan
    with pytest.raises(native.SkylineError) as e:
        ctx.skyline_batch([(good, None), (bad, None)])
    assert e.value.status == native.SKY_EINVAL
    with pytest.raises(native.SkylineError):
        ctx.skyline_batch([(good, None), (np.zeros((4, 9), np.float32), None)])
    assert ctx.skyline_batch([(good, None)])[0].shape[0] > 0


def test_autotune_keeps_result_and_improves_or_keeps_time(ctx):
    from paper_2411_14968_gb300 import native
    x = datagen.anticorrelated(60000, 6, 51)
    base = native.make_params(scheme="sliced", p=8, rep="sorted")
    want = ctx.skyline(x, params=base)
    tuned, ms = ctx.autotune(x, base, max_trials=12)
    assert ms > 0
    assert tuned.scheme == base.scheme and tuned.num_partitions == 8 and tuned.rep == base.rep
    assert tuned.dom_block % 32 == 0 and tuned.chunk_max >= tuned.chunk_min > 0
    np.testing.assert_array_equal(ctx.skyline(x, params=tuned), want)


def test_autotune_batch_keeps_results(ctx):
    from paper_2411_14968_gb300 import native
    xs = [datagen.anticorrelated(40000, 6, 61), datagen.anticorrelated(25000, 5, 62)]
    ps = [native.make_params(scheme="sliced", p=8), native.make_params(scheme="angular", slices=[2, 2, 2, 2])]
    want = [ctx.skyline(x, params=p) for x, p in zip(xs, ps)]
    knobs, ms = ctx.autotune_batch(list(zip(xs, ps)), max_trials=16)
    assert ms > 0 and knobs["dom_block"] % 32 == 0 and knobs["chunk_max"] >= knobs["chunk_min"] > 0
    # the launch shape (tile width, warps per CTA) is one of the compiled ones
    assert knobs["engine_warps"] in (4, 8) and knobs["engine_cands"] in (2, 4)
    tuned = [native.make_params(scheme="sliced", p=8, **knobs),
             native.make_params(scheme="angular", slices=[2, 2, 2, 2], **knobs)]
    for g, w in zip(ctx.skyline_batch(list(zip(xs, tuned))), want):
        np.testing.assert_array_equal(g, w)


def test_graph_replay_matches_and_reads_inputs_at_replay(ctx, oracle_mod):
    import torch
    from paper_2411_14968_gb300 import native
    O = oracle_mod
    x0 = [datagen.anticorrelated(40000, 6, 71), datagen.independent(20000, 4, 72)]
    x1 = [datagen.anticorrelated(40000, 6, 73), datagen.independent(20000, 4, 74)]
    ps = [native.make_params(scheme="sliced", p=8, rep="sorted"), native.make_params(scheme="grid", slices=[3] * 4)]
    ops = [dict(scheme=O.SLICED, p=8, rep=O.REP_SORTED), dict(scheme=O.GRID, slices=[3] * 4)]
    # the expected sets are the oracle's (Algorithm 2 with the same options)
    want0 = [O.partitioned(x, **kw)["indices"] for x, kw in zip(x0, ops)]
    want1 = [O.partitioned(x, **kw)["indices"] for x, kw in zip(x1, ops)]
    xt = [torch.from_numpy(x).cuda() for x in x0]
    g = ctx.capture(list(zip(xt, ps)))
    for _ in range(2):
        res, ms = g.run()
        assert ms > 0
        for r, w in zip(res, want0):
            np.testing.assert_array_equal(r.cpu().numpy().astype(np.uint32), w)
    # inputs rewritten in place: the replay reads them when it runs
    for t, x in zip(xt, x1):
        t.copy_(torch.from_numpy(x))
    res, _ = g.run()
    for r, w in zip(res, want1):
        np.testing.assert_array_equal(r.cpu().numpy().astype(np.uint32), w)
    g.close()
    with pytest.raises(ValueError):
        ctx.capture([(x0[0], ps[0])])
