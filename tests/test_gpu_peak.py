"""The measured FP32 FMA rate (reg_fp32_peak) is physically possible: the best of three
measurements lies above half and below the rate of 128 FP32 lanes per SM at 2.2 GHz (above
the part's maximum SM clock), and no measurement exceeds that bound or falls far below the
best (the first may run while the clocks ramp up from idle)."""
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
    runs = [fp32_peak() for _ in range(3)]
    rates = [tf for tf, _ in runs]
    best = max(rates)
    assert 0.5 * bound < best < bound, (rates, bound)
    assert all(0.5 * best < tf <= best for tf in rates), rates
    assert all(ms > 0.0 for _, ms in runs)
