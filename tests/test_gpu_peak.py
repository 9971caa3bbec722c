"""The measured FP32 FMA rate (reg_fp32_peak) is physically possible: above half and
below the rate of 128 FP32 lanes per SM at 2.2 GHz (above the part's maximum SM clock),
and repeatable."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fp32_peak_is_plausible_and_repeatable():
    import torch
    from paper_1503_00757_gb300.binding import fp32_peak
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    tf1, ms1 = fp32_peak()
    tf2, _ = fp32_peak()
    assert 0.5 * bound < tf1 < bound, (tf1, bound)
    assert 0.5 * bound < tf2 < bound, (tf2, bound)
    assert abs(tf1 - tf2) < 0.1 * max(tf1, tf2)
    assert ms1 > 0.0
