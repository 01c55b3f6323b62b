"""The measurement helper behind the bench's `sfu` record: the device's FP32 exp2 throughput.

Bounds, not a value: at least one exp2 a clock on every SM (a broken or optimised-away kernel
reports far less or absurdly more) and at most 64 a clock and SM at 3 GHz (twice the SFU
width of the part)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ex2_rate_is_a_plausible_sfu_throughput():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_01559_gb300 import binding
    with binding.Context(0) as ctx:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        rate = ctx.measure_ex2_rate()
    assert sms * 1.0e9 <= rate <= sms * 64 * 3.0e9, rate
