"""Measurement support (vmo_measure_alu_peaks): the FP32 rates the step
kernel's roofline is reported against.  The SM count is the device's, the
rates are positive and below the ceiling the SM count and clock allow (128
FP32 lanes per SM, two flops per fused multiply-add), the packed and scalar
fma rates agree (packing halves the instructions, not the pipe's lanes), and
the reciprocal square root, a special-function unit op, runs slower."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4490_gb300 as P
    assert torch.cuda.is_available()
    return P


def test_alu_peaks(V):
    r = V.vmo.measure_alu_peaks()
    props = torch.cuda.get_device_properties(0)
    assert r["sms"] == props.multi_processor_count
    ceiling = r["sms"] * 128 * 2 * 2.2e9 / 1e12  # above any boost clock of the part
    for key in ("ffma_tflops", "ffma2_tflops"):
        assert 0.2 * ceiling < r[key] <= ceiling, (key, r)
    assert 0.7 < r["ffma2_tflops"] / r["ffma_tflops"] < 1.4, r
    assert 0 < r["rsqrt_tops"] < r["ffma_tflops"] / 2, r
