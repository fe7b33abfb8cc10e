"""Serving with continuous batching (sky_submit / sky_wait): requests that
arrive while others are on the GPU join later batches; every result must be
the same as the query's result alone (bit-exact: the result is an index
set), whatever it was batched with."""
import threading
import time

import numpy as np
import pytest

from paper_2411_14968_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_14968_gb300 import native
    return native


def _trace(native, num, seed, n_hi=60000):
    rng = np.random.default_rng(seed)
    qs = []
    schemes = [dict(), dict(scheme="sliced", p=8), dict(scheme="random", p=16, seed=3, rep="sorted"),
               dict(scheme="angular", slices=None), dict(scheme="sliced", p=4, merge="noseq")]
    for i in range(num):
        n = int(10 ** rng.uniform(2, np.log10(n_hi)))
        d = int(rng.integers(3, 9))
        kind = "anticorrelated" if rng.random() < 0.5 else "independent"
        x = datagen.make(kind, n, d, 1000 + i)
        kw = dict(schemes[i % len(schemes)])
        if kw.get("scheme") == "angular":
            kw["slices"] = [2] * (d - 1)
        qs.append((x, native.make_params(**kw)))
    return qs


def test_results_same_alone_and_in_the_mix(native_mod):
    native = native_mod
    qs = _trace(native, 48, 5)
    with native.Context(0) as ctx:
        alone = [ctx.skyline(x, params=p) for x, p in qs]
    with native.Context(0) as ctx:
        ctx.serve_start(workers=2, max_batch=8)
        tickets = [None] * len(qs)

        def client(k):
            # two clients, arrivals spread so that queries arrive while
            # earlier batches are on the GPU
            rng = np.random.default_rng(k)
            for i in range(k, len(qs), 2):
                tickets[i] = ctx.submit(*qs[i])
                time.sleep(float(rng.exponential(0.002)))

        th = [threading.Thread(target=client, args=(k,)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        infos = []
        for i, t in enumerate(tickets):
            got, info = ctx.wait(t)
            infos.append(info)
            np.testing.assert_array_equal(got, alone[i], err_msg=f"query {i}")
        ctx.serve_stop()
    # the loop batched some queries together and ran more than one batch
    assert max(i["batch_queries"] for i in infos) > 1
    assert min(i["batch_queries"] for i in infos) < len(qs)
    assert all(i["latency_us"] >= i["run_us"] >= 0 for i in infos)


def test_restart_after_stop(native_mod):
    # stop and start again, with two workers (whose engine launches are
    # ordered by a gate that must not outlive the stopped workers)
    native = native_mod
    qs = [(datagen.anticorrelated(5000 + 3000 * i, 4 + i % 4, 80 + i), native.make_params(scheme="sliced", p=4))
          for i in range(6)]
    with native.Context(0) as ctx:
        alone = [ctx.skyline(x, params=p) for x, p in qs]
        for workers, mb in ((2, 4), (1, 1), (2, 64), (2, 2)):
            ctx.serve_start(workers=workers, max_batch=mb)
            ts = [ctx.submit(x, p) for x, p in qs]
            for t, want in zip(ts, alone):
                np.testing.assert_array_equal(ctx.wait(t)[0], want)
            ctx.serve_stop()


def test_admission_by_device_memory(native_mod):
    native = native_mod
    qs = [(datagen.anticorrelated(20000, 6, 70 + i), native.make_params(scheme="sliced", p=4)) for i in range(12)]
    with native.Context(0) as ctx:
        alone = [ctx.skyline(x, params=p) for x, p in qs]
        # a budget that holds two of these queries, not three
        one = native.query_bytes(20000, 6, qs[0][1])
        assert one > 20000 * 6 * 4
        ctx.serve_start(workers=1, max_batch=64, mem_budget_bytes=int(2.5 * one))
        ts = [ctx.submit(x, p) for x, p in qs]
        res = [ctx.wait(t) for t in ts]
        for (got, info), want in zip(res, alone):
            np.testing.assert_array_equal(got, want)
            assert info["batch_queries"] <= 2
        ctx.serve_stop()


def test_errors_are_per_ticket(native_mod):
    native = native_mod
    good = datagen.independent(3000, 4, 1)
    bad = good.copy()
    bad[7, 2] = np.nan
    with native.Context(0) as ctx:
        want = ctx.skyline(good)
        ctx.serve_start(workers=1, max_batch=4)
        t1, t2, t3 = ctx.submit(good), ctx.submit(bad), ctx.submit(good)
        np.testing.assert_array_equal(ctx.wait(t1)[0], want)
        with pytest.raises(native.SkylineError) as e:
            ctx.wait(t2)
        assert e.value.status == native.SKY_EINVAL
        np.testing.assert_array_equal(ctx.wait(t3)[0], want)
        # a collected ticket is gone
        with pytest.raises(native.SkylineError) as e:
            ctx.poll(t1)
        assert e.value.status == native.SKY_ECANCELLED
        with pytest.raises(native.SkylineError):
            ctx.submit(np.zeros((5, 9), np.float32))
        ctx.serve_stop()


def test_per_ticket_statistics(native_mod):
    # sky_get_stats(ctx, ticket, ...): a served query's own sizes and counts,
    # equal to what the same query reports when run alone
    native = native_mod
    qs = _trace(native, 12, 7)
    alone = []
    with native.Context(0) as ctx:
        for x, p in qs:
            r = ctx.skyline(x, params=p)
            alone.append((r, ctx.stats()))
    with native.Context(0) as ctx:
        ctx.set_timing(True)
        ctx.serve_start(workers=2, max_batch=4)
        tickets = [ctx.submit(x, p) for x, p in qs]
        for i, t in enumerate(tickets):
            got, info = ctx.wait(t)
            st = ctx.stats(t)  # still available after the ticket is collected
            want, ws = alone[i]
            np.testing.assert_array_equal(got, want)
            assert st["n"] == qs[i][0].shape[0] and st["d"] == qs[i][0].shape[1]
            assert st["skyline"] == want.shape[0]
            for key in ("partitions", "nonempty_partitions", "local_union", "rep_dropped", "grid_dropped",
                        "reps_kept"):
                assert st[key] == ws[key], (i, key)
            assert st["launches"] > 0 and st["ms_total"] > 0
        with pytest.raises(native.SkylineError) as e:
            ctx.stats(tickets[-1] + 1000)
        assert e.value.status == native.SKY_ECANCELLED
        ctx.serve_stop()
