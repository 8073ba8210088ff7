"""p3t_alu_peaks: the measured FP32 FMA and rsqrt ceilings must lie below
the nominal rates (SMs x 128 FP32 lanes x 2 flops, SMs x 16 MUFU lanes, at
the maximum SM clock) and within a factor of two of them; a loop the
compiler dropped would read far above, a broken launch far below."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible(cuda):
    import torch
    import paper_1506_04553_b300 as P
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    clk_hz = 2.032e9  # maximum SM clock of the B300
    fma_nominal = sms * 128 * 2 * clk_hz
    rsqrt_nominal = sms * 16 * clk_hz
    pk = P.alu_peaks()
    for k in ("fma_flops", "fma2_flops"):
        assert 0.5 * fma_nominal < pk[k] < 1.05 * fma_nominal, (k, pk[k], fma_nominal)
    assert 0.5 * rsqrt_nominal < pk["rsqrt_ops"] < 1.05 * rsqrt_nominal, pk


def test_fp64_peaks_are_plausible(cuda):
    """FP64 FMA/s between a quarter and the nominal rate of the B300 (about
    2 FP64 lanes per clock per SM); a dependent add takes at least a few
    cycles, and a correctly rounded division or square root (several
    dependent FMAs) takes longer than an add."""
    import torch
    import paper_1506_04553_b300 as P
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 2.1 * 2.032e9
    pk = P.fp64_peaks()
    assert 0.25 * nominal < pk["dfma_ops"] < 1.1 * nominal, (pk, nominal)
    assert 4 <= pk["add_cycles"] < 2000, pk
    assert pk["div_cycles"] > 2 * pk["add_cycles"], pk
    assert pk["sqrt_cycles"] > 2 * pk["add_cycles"], pk
