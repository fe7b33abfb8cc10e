"""The measurement probes of include/skyline_diag.h (roofline denominators):
they run on every SM of the device and report a positive rate, and refuse
zero iterations."""
import pytest

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


def test_probes_report_rates(ctx):
    import torch
    from paper_2411_14968_gb300 import native
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for probe in (ctx.probe_compare_rate, ctx.probe_reject_rate):
        rate, n = probe(50)
        assert n == sms
        # between 1e12 and 1e15 compares per second on any current GPU
        assert 1e12 < rate < 1e15
        with pytest.raises(native.SkylineError) as e:
            probe(0)
        assert e.value.status == native.SKY_EINVAL
