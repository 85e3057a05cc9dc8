"""The FMA-rate probe (roofline denominator of the FP64 passes) on the GPU:
rates must lie near what the SM count and clock allow (FP64: 2 FMA lanes per
SM, FP32: 128), and an unsupported precision is rejected."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible():
    import paper_1104_5330_gb300.ts as T
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceil64 = sms * 2 * 2 * 2.2e9 / 1e12          # above any boost clock
    ceil32 = sms * 2 * 128 * 2.2e9 / 1e12
    r64 = T.ts_probe_fma_rate(T.TS_FP64)
    r32 = T.ts_probe_fma_rate(T.TS_FP32)
    assert 0.2 * ceil64 < r64 < ceil64, r64
    assert 0.2 * ceil32 < r32 < ceil32, r32
    with pytest.raises(T.TSError):
        T.ts_probe_fma_rate(T.TS_TF32X3)
