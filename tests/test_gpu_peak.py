"""The FMA-loop peak entry point (instrumentation: the denominator of the
roofline fraction of the FP64-pipe-bound kernels)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def test_fma_peaks_are_plausible_for_the_device(dgmg):
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fp64 = dgmg.fma_peak(0)
    fp32 = dgmg.fma_peak(1)
    fp32x2 = dgmg.fma_peak(2)
    # upper bounds from the SM count at a 3 GHz ceiling: 64 FP64 and 256 FP32
    # lanes per SM are more than any part of this family has
    assert 0.0 < fp64 <= sms * 64 * 2 * 3.0e9 / 1e12
    assert 0.0 < fp32 <= sms * 256 * 2 * 3.0e9 / 1e12
    assert 0.0 < fp32x2 <= sms * 256 * 2 * 3.0e9 / 1e12
    assert fp32 > 10.0 * fp64
    assert dgmg.wait_timeouts() == 0


def test_fma_peak_rejects_unknown_kinds(dgmg):
    with pytest.raises(dgmg.DGMGError) as ei:
        dgmg.fma_peak(3)
    assert ei.value.code == dgmg.DGMG_EINVAL
