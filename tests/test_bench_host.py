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


def test_traffic_record_from_an_ncu_csv(tmp_path):
    """The record is parsed from the capture's CSV (base units), the traffic
    is read + write, and the stamp is the hash of the current sources, which
    is what makes bench.py report the record's traffic."""
    csv = tmp_path / "traffic.csv"
    csv.write_text(
        '==PROF== Connected to process 1\n'
        '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
        '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
        '"0","1","python","h","void geo::rr_kernel<A, 8, true>(geo::TileLaunch)","1","7","(512, 1, 1)",'
        '"(144, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","2,212,352"\n'
        '"0","1","python","h","void geo::rr_kernel<A, 8, true>(geo::TileLaunch)","1","7","(512, 1, 1)",'
        '"(144, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","370,432"\n'
        '"0","1","python","h","void geo::rr_kernel<A, 8, true>(geo::TileLaunch)","1","7","(512, 1, 1)",'
        '"(144, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","nsecond","713,000"\n')
    out = tmp_path / "rec.json"
    rec = bench.write_traffic_record(str(csv), str(out))
    assert rec["traffic_bytes_per_launch"] == 2212352 + 370432
    assert rec["gpu_time_ms_under_ncu"] == pytest.approx(0.713)
    assert rec["source_sha256"] == bench.kernel_source_sha256()
    assert "rr_kernel" in rec["kernel"]
