"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Dominance is exact comparison arithmetic and the partition indices are
integer or single-rounding FP32 definitions, so the bar is bit-exactness:
the skyline index set, every point's partition and every point's stage code
(where it left Algorithm 2) must equal the oracle's."""
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


def _oracle_kw(scheme, p, slices, normalize, rep, merge, seed=0, slice_dim=0, grid_filter=True):
    from oracle import oracle as O
    return dict(scheme={"random": O.RANDOM, "grid": O.GRID, "angular": O.ANGULAR, "sliced": O.SLICED,
                        "none": O.NONE}[scheme], p=p, slices=slices, normalize=normalize, seed=seed,
                rep={"none": 0, "sorted": 1, "region": 2}[rep], merge={"sequential": 0, "noseq": 1}[merge],
                slice_dim=slice_dim, grid_filter=grid_filter)


def _check(ctx, oracle_mod, x, scheme="none", p=1, slices=None, normalize=False, rep="none",
           merge="sequential", exec="persistent", seed=0, slice_dim=0, reps_per_partition=1, **tune):
    want = oracle_mod.partitioned(x, reps_per_partition=reps_per_partition,
                                  **_oracle_kw(scheme, p, slices, normalize, rep, merge, seed, slice_dim))
    idx, pid, stage = ctx.skyline(x, scheme=scheme, p=p, slices=slices, normalize=normalize, rep=rep,
                                  merge=merge, exec=exec, seed=seed, slice_dim=slice_dim, with_diag=True,
                                  reps_per_partition=reps_per_partition, **tune)
    tag = f"{scheme} p={p} slices={slices} rep={rep} merge={merge} exec={exec}"
    np.testing.assert_array_equal(idx, want["indices"], err_msg=tag)
    np.testing.assert_array_equal(pid, want["pid"], err_msg=tag + " pid")
    np.testing.assert_array_equal(stage, want["stage"], err_msg=tag + " stage")
    if x.shape[0]:
        st = ctx.stats()
        assert st["nonempty_partitions"] == np.unique(want["pid"]).shape[0], tag
        assert st["skyline"] == want["indices"].shape[0], tag
    return idx


# The tiny workload: N = 10,000 anticorrelated, d = 4, Grid m = 2 per dimension.
def test_tiny_grid_anticorrelated(ctx, oracle_mod):
    x = datagen.anticorrelated(10000, 4, 1)
    for rep in ("none", "sorted"):
        for merge in ("sequential", "noseq"):
            for ex in ("persistent", "plain"):
                _check(ctx, oracle_mod, x, "grid", slices=[2, 2, 2, 2], rep=rep, merge=merge, exec=ex)


VARIANTS = [
    ("none", 1, None),
    ("random", 16, None),
    ("sliced", 8, None),
    ("grid", 1, "g"),
    ("angular", 1, "a"),
]


@pytest.mark.parametrize("kind", ["anticorrelated", "independent", "correlated", "skewed"])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_all_schemes(ctx, oracle_mod, kind, d):
    x = datagen.make(kind, 3000, d, 100 + d)
    norm = kind == "skewed"
    for scheme, p, sl in VARIANTS:
        slices = None
        if sl == "g":
            slices = [2] * d if d > 2 else [5] * d
        elif sl == "a":
            if d == 1:
                continue
            slices = ([4, 3, 2, 2, 2, 2, 2])[: d - 1]
        for rep in ("none", "sorted", "region"):
            for merge in ("sequential", "noseq"):
                _check(ctx, oracle_mod, x, scheme, p, slices, norm, rep, merge, seed=7)


def test_several_representatives_per_partition(ctx, oracle_mod):
    # k > 1 Sorted and Region representatives (Section 4.1), with ties of
    # volume (quantised data) broken by index, and normalised volumes on data
    # outside [0, 1]
    x = datagen.independent(20000, 4, 21)
    y = datagen.make("skewed", 8000, 5, 22)
    for rep in ("sorted", "region"):
        for k in (2, 7):
            _check(ctx, oracle_mod, x, "sliced", 9, rep=rep, reps_per_partition=k)
            _check(ctx, oracle_mod, y, "random", 5, normalize=True, rep=rep, reps_per_partition=k, seed=3)
    _check(ctx, oracle_mod, y, "angular", 1, [3, 2, 2, 2], normalize=False, rep="region", reps_per_partition=3)


def test_multi_round_small_chunks(ctx, oracle_mod):
    # small chunks and dominator blocks force many SFS rounds, many window
    # blocks and ragged tails in every partition
    x = datagen.anticorrelated(20000, 5, 3)
    for scheme, p, sl in (("none", 1, None), ("sliced", 5, None), ("angular", 1, [3, 2, 2, 2])):
        for ex in ("persistent", "plain"):
            _check(ctx, oracle_mod, x, scheme, p, sl, exec=ex, chunk_min=96, chunk_max=700,
                   chunk_alpha_x4=3, dom_block=64)


def test_engine_tiles_and_blocks(ctx, oracle_mod):
    # chunks of several candidate tiles, dense lists of several tiles, one or
    # many window blocks per round
    x = datagen.anticorrelated(60000, 6, 11)
    for scheme, p, sl in (("none", 1, None), ("sliced", 3, None)):
        for db in (128, 2048):
            _check(ctx, oracle_mod, x, scheme, p, sl, chunk_min=3000, chunk_max=9000, dom_block=db)


def test_fp16_image_collisions(ctx, oracle_mod):
    # The engine rejects pairs on FP16 round-down images before the FP32
    # test.  (a) every attribute in [1, 1 + 2^-10): all points share one FP16
    # image, so FP32 decides every test; (b) magnitudes beyond the FP16 range
    # (the images are clamped to +-65504) and negative values; (c) values of
    # both signs around the FP16 subnormal range, where the images and their
    # differences are subnormal or zero.
    rng = np.random.default_rng(12)
    n = 4000
    a = (1.0 + rng.integers(0, 512, (n, 4)) * 2.0 ** -23).astype(np.float32)
    b = (rng.standard_normal((n, 5)) * 1e6).astype(np.float32)
    b[::7, 2] = np.float32(3e38)
    b[::11, 1] = np.float32(-3e38)
    b[::13, 4] = np.float32(70000.0)
    b[::17, 4] = np.float32(65504.0)
    c = (rng.standard_normal((n, 6)) * 2e-7).astype(np.float32)
    c[::9, 3] = np.float32(5.96e-8)
    c[::10, 0] = np.float32(-5.96e-8)
    for x in (a, b, c):
        for scheme, p in (("none", 1), ("sliced", 4), ("random", 8)):
            _check(ctx, oracle_mod, x, scheme, p, rep="sorted", dom_block=128)
            _check(ctx, oracle_mod, x, scheme, p, merge="noseq")


def test_quantised_ties(ctx, oracle_mod):
    # many equal scores and exact duplicates: chunk cuts must not split runs
    for kind in ("independent", "correlated"):
        x = datagen.make(kind, 30000, 8, 5)
        x = (np.floor(x * 8) / 8).astype(np.float32)
        for scheme, p, sl in (("none", 1, None), ("grid", 1, [2] * 8), ("random", 32, None)):
            _check(ctx, oracle_mod, x, scheme, p, sl, rep="sorted", chunk_min=128, dom_block=96)


def test_edge_values(ctx, oracle_mod):
    rng = np.random.default_rng(4)
    x = rng.random((4000, 3)).astype(np.float32)
    x[:100] = 0.0
    x[100:200] = -0.0
    x[200:260, 1] = np.inf
    x[260:300, 0] = -np.inf
    x[300:340] = np.float32(1e-45)  # denormals: no flush to zero
    x[340:380, 2] = np.float32(2e-45)
    x[400:800] = x[800:1200]        # duplicates
    for scheme, p, sl in VARIANTS:
        slices = [3, 3, 3] if sl == "g" else ([3, 2] if sl == "a" else None)
        _check(ctx, oracle_mod, x, scheme, p, slices, rep="sorted", merge="noseq")
        _check(ctx, oracle_mod, x, scheme, p, slices, rep="none", merge="sequential")


def test_small_n(ctx, oracle_mod):
    for n in (1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 129):
        x = datagen.independent(n, 4, n)
        for scheme, p, sl in VARIANTS:
            slices = [2, 2, 2, 2] if sl == "g" else ([2, 2, 2] if sl == "a" else None)
            _check(ctx, oracle_mod, x, scheme, p, slices, rep="sorted", merge="noseq")


def test_empty_and_all_equal(ctx):
    x = np.zeros((0, 5), np.float32)
    assert ctx.skyline(x).shape == (0,)
    y = np.full((5000, 6), 0.5, np.float32)
    np.testing.assert_array_equal(ctx.skyline(y, scheme="sliced", p=7), np.arange(5000))


def test_device_tensor_input(ctx, oracle_mod):
    import torch
    x = datagen.anticorrelated(50000, 6, 9)
    want = oracle_mod.partitioned(x, scheme=oracle_mod.SLICED, p=16)["indices"]
    t = torch.from_numpy(x).cuda()
    got = ctx.skyline(t, scheme="sliced", p=16, rep="sorted")
    assert got.is_cuda
    np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint32), want)


def test_invalid_inputs(ctx):
    from paper_2411_14968_gb300 import native
    x = datagen.independent(100, 3, 1)
    x[17, 1] = np.nan
    with pytest.raises(native.SkylineError) as e:
        ctx.skyline(x)
    assert e.value.status == native.SKY_EINVAL
    with pytest.raises(native.SkylineError):
        ctx.skyline(np.zeros((10, 9), np.float32))
    with pytest.raises(native.SkylineError):
        ctx.skyline(datagen.independent(10, 3, 1), scheme="sliced", p=2, slice_dim=3)
    # the context stays usable after errors
    assert ctx.skyline(datagen.independent(100, 3, 1)).shape[0] > 0


# Every compiled launch shape of the engine (warps per CTA x candidates per
# lane: the tile width of a work item) gives the oracle's result, with the
# default knobs and with small chunks and blocks that force many rounds.
@pytest.mark.parametrize("warps,cands", [(4, 4), (8, 4), (4, 2), (8, 2)])
def test_engine_launch_shapes(ctx, oracle_mod, warps, cands):
    shape = dict(engine_warps=warps, engine_cands=cands)
    x6 = datagen.anticorrelated(20011, 6, 81)
    _check(ctx, oracle_mod, x6, "sliced", p=8, **shape)
    _check(ctx, oracle_mod, x6, "angular", slices=[2, 2, 2, 1, 1], rep="sorted", merge="noseq", **shape)
    _check(ctx, oracle_mod, x6, "random", p=5, seed=3, chunk_min=256, chunk_max=1024, dom_block=256, **shape)
    x8 = datagen.independent(30001, 8, 82)
    _check(ctx, oracle_mod, x8, "grid", slices=[2] * 8, **shape)
    x3 = datagen.correlated(9001, 3, 83, quantised=False)
    _check(ctx, oracle_mod, x3, "none", exec="plain", **shape)
    _check(ctx, oracle_mod, x3[:1], "none", **shape)


def test_engine_launch_shape_rejected(ctx):
    from paper_2411_14968_gb300 import native
    x = datagen.anticorrelated(1000, 4, 84)
    for bad in (dict(engine_warps=2), dict(engine_cands=3), dict(engine_warps=16, engine_cands=4)):
        with pytest.raises(native.SkylineError) as e:
            ctx.skyline(x, **bad)
        assert e.value.status == native.SKY_EINVAL


# Local launches of more than eight segments keep each round's dense list in
# score order by last-tile compaction while the round's chunk is at most 16k
# points, and fall back to arrival order for longer chunks: segments of 25k
# and 30k points reach both within one launch; both must give the oracle's
# partitions, stage codes and skyline.
def test_local_dense_list_modes(ctx, oracle_mod):
    x = datagen.anticorrelated(300000, 5, 85)
    _check(ctx, oracle_mod, x, "sliced", p=12)
    _check(ctx, oracle_mod, x, "random", p=10, seed=4, rep="sorted")
    _check(ctx, oracle_mod, x, "sliced", p=12, chunk_min=4096, chunk_alpha_x4=64)


def test_engine_test_counts(ctx, oracle_mod):
    """sky_stats counts the engine's dominance tests: every point the engine
    removed (stage 4, and stage 5 under the sequential merge) took at least
    one, the local phase's are part of the total, and with NoSeq (no merge
    in the engine) they are all of it."""
    from paper_2411_14968_gb300 import native
    x = datagen.anticorrelated(20000, 4, 5)
    for merge in ("sequential", "noseq"):
        for ex in ("persistent", "plain"):
            _, _, stage = ctx.skyline(x, scheme="sliced", p=8, merge=merge, exec=ex, with_diag=True)
            st = ctx.stats()
            kills = int((stage == native.STAGE_LOCAL).sum())
            if merge == "sequential":
                kills += int((stage == native.STAGE_MERGE).sum())
            assert st["tests_fp16"] >= kills > 0, (merge, ex, st["tests_fp16"], kills)
            assert 0 < st["tests_fp16_local"] <= st["tests_fp16"]
            if merge == "noseq":
                assert st["tests_fp16_local"] == st["tests_fp16"]
            else:
                assert st["tests_fp16_local"] < st["tests_fp16"]
    # a batch reports the tests of all its launches; a query of the shared
    # launches reports theirs
    ps = [native.make_params(scheme="sliced", p=8), native.make_params(scheme="grid", slices=[2] * 4)]
    ctx.skyline_batch([(x, p) for p in ps])
    st = ctx.stats()
    ctx.skyline(x, params=ps[0])
    alone = ctx.stats()
    assert st["tests_fp16"] > alone["tests_fp16"] > 0
