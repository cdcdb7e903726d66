"""The measured FP32 FMA rate (the fused kernel's second roofline
denominator) is positive and no higher than the nominal peak at the
device's maximum clock: SMs x 128 lanes x 2 flops x 2070 MHz."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1408_6373_gb300 as cg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


def test_fma_rate_within_nominal(ctx):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2070e6 / 1e12
    tflops, ms = ctx.fp32_fma_rate()
    assert ms > 1.0
    assert 0.2 * nominal < tflops <= 1.02 * nominal
