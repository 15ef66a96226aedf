"""The FMA-rate probe (gr_fma_rate): positive, finite rates, FP32 well above
FP64 on this part (FP64 FMAs issue at a small fraction of the FP32 rate), and
both below the rate that the SMs' unit counts at the maximum clock allow."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr  # noqa: E402


def test_fma_rates():
    f64 = gr.gr_fma_rate(True, 1 << 14)
    f32 = gr.gr_fma_rate(False, 1 << 14)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # FMA units per SM: 128 FP32 (every CUDA-capable SM since Volta has at least 64); FP64 at most 64
    # per SM on any part; clocks below 3 GHz
    assert 0 < f64 < sms * 64 * 2 * 3e9
    assert 0 < f32 < sms * 128 * 2 * 3e9
    assert f32 > 4 * f64
