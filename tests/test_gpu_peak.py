"""The integer-pipe probe that gives the roofline its denominator."""
import pytest

pytestmark = pytest.mark.gpu


def test_int_peak_is_plausible_and_scales_with_work():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    r1, ms1 = sg.sogrand_int_peak(20_000)
    r2, ms2 = sg.sogrand_int_peak(40_000)
    # GB300: 152 SMs at up to ~2.1 GHz; between 16 and 512 lane-ops per SM and clock
    for r in (r1, r2):
        assert 152 * 16 * 1.0e9 < r < 152 * 512 * 2.2e9
    assert 1.6 < ms2 / ms1 < 2.4  # twice the trips, about twice the time
    with pytest.raises(sg.SograndError):
        sg.sogrand_int_peak(0)
