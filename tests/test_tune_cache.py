"""The autotuner's JSON cache of tuned knobs (host side, no GPU): keys
separate workload shapes and method parameters but not the knobs, and
entries survive a round trip through the file."""
import json

from paper_2411_14968_gb300 import native


def test_tune_key_shapes_and_parameters():
    p = native.make_params(scheme="sliced", p=64)
    k = native.tune_key(1_000_000, 6, p)
    assert k == native.tune_key(1_000_000, 6, native.make_params(scheme="sliced", p=64))
    # N is bucketed by powers of two
    assert native.tune_key(600_000, 6, p) == k and native.tune_key(1 << 20, 6, p) != k
    assert native.tune_key(1_000_000, 5, p) != k
    for other in (dict(scheme="sliced", p=32), dict(scheme="sliced", p=64, rep="sorted"),
                  dict(scheme="sliced", p=64, merge="noseq"), dict(scheme="sliced", p=64, images="ranks")):
        assert native.tune_key(1_000_000, 6, native.make_params(**other)) != k, other
    # the knobs themselves are not part of the key
    q = native.make_params(scheme="sliced", p=64, chunk_min=4096, dom_block=512, engine_warps=8)
    assert native.tune_key(1_000_000, 6, q) == k
    assert json.loads(k)["log2_n"] == 19


def test_tune_cache_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    c = native.TuneCache(str(path))
    assert c.get("x") is None
    tuned = native.make_params(scheme="grid", slices=[2] * 4, chunk_min=256, chunk_max=65536, chunk_alpha_x4=16,
                               dom_block=2048, engine_warps=8, engine_cands=2)
    key = native.tune_key(10_000, 4, tuned)
    c.put(key, tuned, 1.25)
    again = native.TuneCache(str(path))
    entry = again.get(key)
    assert entry["ms"] == 1.25
    fresh = native.TuneCache.apply(entry, native.make_params(scheme="grid", slices=[2] * 4))
    for k in native.KNOBS:
        assert getattr(fresh, k) == getattr(tuned, k), k
    assert fresh.scheme == native.SCHEMES["grid"]
