"""The FMA-rate diagnostic returns the device's FP32 and FP64 issue rates:
FP32 within the unit-count bound (SMs x 128 lanes x 2 flop x clock) and
above a third of it; FP64 positive and far below FP32 on this part."""
import pytest
import torch

from paper_1808_02281_gb300 import build as B
from paper_1808_02281_gb300 import lqcd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def test_fma_rates():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12     # 2.2 GHz: above any boost clock of the part
    f32 = lqcd.measure_fma_rate("f32")
    f64 = lqcd.measure_fma_rate("f64")
    assert bound / 3 < f32 <= bound, (f32, bound)
    assert 0.0 < f64 < f32, (f64, f32)
