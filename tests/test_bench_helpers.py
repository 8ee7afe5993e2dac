"""Host-side helpers of bench.py that need no GPU: the algorithmic flop
counts and peaks the roofline objects divide by, and the oracle's ANCF
baseline sample."""
import pytest

import bench


def test_ancf_flop_counts():
    """47,184 / 604,776 flop per beam / shell element for the assembly pass and
    11,940 / 88,464 for the force pass (counts stated in the bench's comment:
    per point 100n + 183, force 21 n per point, tangent 77 per pair and point,
    mass 3 per pair)."""
    assert bench.ancf_flops_per_elem("ancf3243") == 12 * (100 * 8 + 183) + 21 * 8 * 12 + 36 * 12 * 77 + 3 * 36
    assert bench.ancf_flops_per_elem("ancf3243") == 47_184
    assert bench.ancf_flops_per_elem("ancf3443") == 604_776
    assert bench.ancf_flops_per_elem("ancf3243", tangent=False) == 11_940
    assert bench.ancf_flops_per_elem("ancf3443", tangent=False) == 88_464


def test_alu_peaks():
    """Derived ALU peaks: 152 SMs at 2.07 GHz, 128 float32 lanes or 2 float64
    FMA per SM and clock, 2 flop per FMA."""
    assert bench.fp32_alu_peak_tflops() == pytest.approx(80.54784)
    assert bench.fp64_alu_peak_tflops() == pytest.approx(1.25856)


@pytest.mark.parametrize("kind,ne", [("ancf3243", 64), ("ancf3443", 16)])
def test_oracle_ancf_rate_sample(kind, ne):
    rate, reps, n, el = bench.oracle_ancf_rate(kind, budget_s=0.05)
    assert n == ne and reps >= 1 and el > 0.0 and rate == pytest.approx(reps * n / el)
