"""sky_skyline_static, the entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc when they need a skyline
(an allocator that owns all device memory, a loop that must not allocate or
synchronise on cudaFree, a fixed memory footprint); its scratch is a
file-scope device array of the library.  The tests call it through the C ABI
and check its output against the CPU oracle and against sky_skyline's, on
two calls in a row -- the second call reuses the array the first left
behind -- at every d, at one point and at the size limit, with -0.0 and
duplicate inputs, on a non-default stream; a NaN is refused and leaves the
next call correct, and sizes beyond the limit are refused.  The file is
named to be collected last."""
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


def _static(torch, x, stream=None):
    from paper_2411_14968_gb300 import native
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if stream is None:
        got = native.skyline_static(xt)
    else:
        with torch.cuda.stream(stream):
            got = native.skyline_static(xt)
    torch.cuda.synchronize()
    return got.cpu().numpy().astype(np.uint32)


def test_static_entry_point_matches_oracle_and_sky_skyline(torch_cuda, oracle_mod):
    from paper_2411_14968_gb300 import native
    torch = torch_cuda
    cases = [datagen.anticorrelated(3001 + 7 * d, d, 20 + d) for d in range(1, 9)]
    dup = datagen.independent(5000, 3, 22)
    dup[:50] = dup[50:100]  # exact duplicates must both stay
    cases.append(dup)
    with native.Context(0) as ctx:
        for x in cases:
            want = oracle_mod.skyline_indices(x)
            np.testing.assert_array_equal(ctx.skyline(x), want)
            for _ in range(2):  # the second call finds the first one's scratch
                np.testing.assert_array_equal(_static(torch, x), want, err_msg=f"d={x.shape[1]}")


def test_static_entry_point_edges(torch_cuda, oracle_mod):
    from paper_2411_14968_gb300 import native
    torch = torch_cuda
    # one point
    np.testing.assert_array_equal(_static(torch, np.array([[0.5, 0.25]], np.float32)), [0])
    # -0.0 equals +0.0: (-0, 1) and (+0, 1) are copies (both kept), and
    # (-0, 0.5) dominates (+0, 1) and its copy
    z = np.array([[-0.0, 1.0], [0.0, 1.0], [1.0, -0.0], [0.0, 0.5], [-0.0, 0.5]], np.float32)
    want = oracle_mod.skyline_indices(z)
    np.testing.assert_array_equal(want, [2, 3, 4])
    np.testing.assert_array_equal(_static(torch, z), want)
    # on a stream of its own, twice
    s = torch.cuda.Stream()
    x = datagen.independent(20000, 5, 31)
    want = oracle_mod.skyline_indices(x)
    for _ in range(2):
        np.testing.assert_array_equal(_static(torch, x, stream=s), want)
    # a NaN is refused, and the next call (same scratch) is still correct
    bad = x.copy()
    bad[777, 2] = np.nan
    with pytest.raises(native.SkylineError) as e:
        _static(torch, bad)
    assert e.value.status == native.SKY_EINVAL
    np.testing.assert_array_equal(_static(torch, x), want)


def test_static_entry_point_at_its_limit(torch_cuda, oracle_mod):
    from paper_2411_14968_gb300 import native
    torch = torch_cuda
    n = native.STATIC_MAX_POINTS
    x = datagen.anticorrelated(n, 8, 23)
    want = oracle_mod.skyline_indices(x)
    with native.Context(0) as ctx:
        np.testing.assert_array_equal(ctx.skyline(x), want)
    for _ in range(2):
        np.testing.assert_array_equal(_static(torch, x), want)
    # sizes beyond the fixed scratch array are refused, not truncated
    big = torch.zeros((n + 1, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(native.SkylineError) as e:
        native.skyline_static(big)
    assert e.value.status == native.SKY_EINVAL
