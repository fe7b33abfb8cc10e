"""The persistent engine's bounded waits end in an error status, not a hang.

Every device-side wait of the engine (for a bulk copy, for the task of a
claimed ticket, for a preceding tile's survivor count) gives up when no work
item anywhere in the launch has completed for a time limit.  The test arms
the context's test hook (include/skyline_diag.h): a 50 ms limit and one
task of the launch that keeps its tickets but is never published, so the
CTAs that draw those tickets wait for a task that never comes.  The call
must return SKY_ETIMEOUT, and the next call on the same context must return
the oracle's skyline."""
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


@pytest.mark.parametrize("withhold", [3, 12])
def test_withheld_task_times_out_and_context_stays_usable(ctx, oracle_mod, withhold):
    from paper_2411_14968_gb300 import native
    x = datagen.anticorrelated(60000, 5, 91)
    kw = dict(scheme="sliced", p=8)
    want = oracle_mod.partitioned(x, scheme=oracle_mod.SLICED, p=8)["indices"]
    np.testing.assert_array_equal(ctx.skyline(x, **kw), want)
    # withhold = 3: a phase A of round 0 (the prologue publishes one task per
    # partition); withhold = 12: a task that a completing tile publishes mid-launch
    ctx.engine_wait_test(50_000_000, withhold)
    with pytest.raises(native.SkylineError) as e:
        ctx.skyline(x, **kw)
    assert e.value.status == native.SKY_ETIMEOUT
    # the hook applied to that call only; the context is still usable
    for _ in range(2):
        np.testing.assert_array_equal(ctx.skyline(x, **kw), want)


def test_wait_test_hook_rejects_bad_limits(ctx):
    from paper_2411_14968_gb300 import native
    with pytest.raises(native.SkylineError) as e:
        ctx.engine_wait_test(1000, 1)
    assert e.value.status == native.SKY_EINVAL
