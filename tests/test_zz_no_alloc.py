"""sky_skyline_static, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc when they need a skyline
(an allocator that owns all device memory, a loop that must not allocate or
synchronise on cudaFree, a fixed memory footprint); its scratch is a
file-scope device array of the library.  The test calls it through the C ABI
and checks its output against sky_skyline's on two calls in a row -- the
second call reuses the array the first left behind -- and that sizes beyond
its limit are refused.  The file is named to be collected last."""
import numpy as np
import pytest

from paper_2411_14968_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_static_entry_point_matches_sky_skyline():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2411_14968_gb300 import native
    cases = [datagen.anticorrelated(30000, 6, 21), datagen.independent(5000, 3, 22)]
    cases[1][:50] = cases[1][50:100]  # exact duplicates must both stay
    with native.Context(0) as ctx:
        for x in cases:
            want = ctx.skyline(x)
            got = native.skyline_static(torch.from_numpy(x).cuda())
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy().astype(np.uint32), want)
    # sizes beyond the fixed scratch array are refused, not truncated
    big = torch.zeros((native.STATIC_MAX_POINTS + 1, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(native.SkylineError) as e:
        native.skyline_static(big)
    assert e.value.status == native.SKY_EINVAL
