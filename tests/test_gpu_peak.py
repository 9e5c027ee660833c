"""The measured multiply-add ceiling (festung_fma_peak) lies between a tenth of and the
nominal rate of the device (152 SMs x 128 FP32 lanes x 2 flop x ~2 GHz ~ 80 TFLOP/s; FP64
at a small fraction of it on GB300)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1408_3877_gb300 import festung as F
    f32, f64 = F.fma_peak(F.FP32), F.fma_peak(F.FP64)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.1 * nominal < f32 <= 1.05 * nominal, (f32, nominal)
    assert 0.0 < f64 < f32, (f64, f32)
