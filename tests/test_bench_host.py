"""Host-side arithmetic of the benchmark line (no GPU): the ALU roofline's
peak from the measured packed min/max rate, and the choice of the faster
probed form."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_peak_from_unit_rate_and_clock():
    # 152 SMs x 64 lane-ops per clock x 2 pixels per packed op x 2070 MHz
    assert bench.alu_peak_top_s(152, 64, 2070.0) == pytest.approx(40.27392, rel=1e-12)
    # the issue-rate figure reported beside it
    assert bench.alu_peak_top_s(152, 128, 2070.0) == pytest.approx(80.54784, rel=1e-12)


def test_probe_takes_the_faster_form():
    class FakeLib:
        def probe_minmax_rate(self, form):
            return {"u16x2": (63.9, 2068.0), "f16x2": (64.1, 2069.0)}[form]

    rate, mhz, form = bench.probe_alu(FakeLib())
    assert (rate, mhz, form) == (64.1, 2069.0, "f16x2")

