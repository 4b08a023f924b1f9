"""The arithmetic-throughput probe (wcns_alu_probe) through the C ABI: FMA
chains on every SM reach a plausible share of the rate derived from the
unit counts (FP32: 128 lanes x 2 flops per SM per clock; FP64: 2 FMA units
x 2 flops), and bad arguments are rejected."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_07806_gb300 import wcns  # noqa: E402


def test_probe_rates_against_unit_counts():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32, packed, fp64 = (wcns.alu_probe(k) for k in range(3))
    # per SM per clock, with clocks between 0.5 and 2.2 GHz
    for rate, per_clock in ((fp32, 256), (fp64, 4)):
        lo, hi = sms * per_clock * 0.5e9 * 0.3 / 1e12, sms * per_clock * 2.2e9 / 1e12
        assert lo < rate < hi, (rate, lo, hi)
    assert packed > 0.5 * fp32
    with pytest.raises(wcns.WcnsError):
        wcns.alu_probe(3)
