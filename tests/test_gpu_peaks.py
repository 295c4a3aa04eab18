"""The FMA-throughput microbenchmark measures what it claims: float32 at or
below the unit-count peak (152 SMs x 128 lanes x 2 flops x the maximum SM
clock, with 5% allowance) and above half of it, and float64 far below
float32 on this part."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    import torch
    from paper_1110_0740_gb300 import ctu
    torch.cuda.init()
    props = torch.cuda.get_device_properties(0)
    f32 = ctu.ctu_fma_peak(0, 1 << 16)
    f64 = ctu.ctu_fma_peak(1, 1 << 12)
    peak32 = props.multi_processor_count * 128 * 2 * 2.07e9
    assert 0.5 * peak32 < f32 <= 1.05 * peak32, (f32, peak32)
    assert 0 < f64 < f32 / 8, (f64, f32)
