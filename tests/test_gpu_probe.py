"""dgs_probe_alu measures plausible issue rates: FP32 FMA throughput within
the range the SM count and clock allow (152 SMs x 128 lanes x 2 FLOP at
1-2.1 GHz), exp2 throughput between 1/16 and 1/2 of the FMA rate."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_alu_rates():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    r = c.probe_alu()
    c.close()
    lanes = r["sm_count"] * 128 * 2
    assert lanes * 0.8e9 / 1e12 <= r["fp32_tflops"] <= lanes * 2.2e9 / 1e12, r
    fma_per_s = r["fp32_tflops"] * 1e12 / 2
    assert fma_per_s / 16 <= r["ex2_per_s"] <= fma_per_s / 2, r
