"""The FP64 FMA probe (the measured denominator of the FP64 rooflines): its rate matches 4 FP64 flops per clock
and SM (2 FMA lanes) at the clock it measured, and its clock is a plausible SM clock."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402


def test_fp64_probe_rate_and_clock():
    torch.cuda.set_device(0)
    ctx = mfa.Context(0, torch.cuda.current_stream())
    tflops, mhz = mfa.mfa_probe_fp64_fma(ctx.h)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 500.0 < mhz < 3000.0, mhz
    per_clock_per_sm = tflops * 1e12 / (sms * mhz * 1e6)
    assert 3.0 < per_clock_per_sm < 4.2, (tflops, mhz, per_clock_per_sm)
