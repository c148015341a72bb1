"""The min/max rate probe behind the benchmark's ALU rooflines."""
import pytest


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["u16x2", "f16x2", "f32x3", "mix"])
def test_probe_reports_a_rate_within_the_issue_limit(form):
    import paper_1911_13074_gb300 as gm
    rate, mhz = gm.probe_minmax_rate(form)
    # a warp scheduler issues at most one instruction per clock: 4 x 32 lanes per SM
    assert 8.0 <= rate <= 128.5
    assert 100.0 <= mhz <= 4000.0
    assert gm.device_status() == 0
