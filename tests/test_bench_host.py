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


def test_dtype_fractions_of_the_secondary_measurements():
    """Each case against its element path's peak: uint8 at 2.5 instructions
    per masked pixel-step (2 unmasked), float32 at 3 (2); float64 chains of
    160 steps or more run the float32 kernel on ranks; reconstructions count
    the plain method's work from the oracle's changing steps."""
    sec = {"workload1_1024": {"workload": "x",
                              "chain_u8_dilate_conn8_steps1500": {"ms": 0.72, "gpixel_steps_per_s": 2000.0},
                              "window_u8_dilate_s13": {"ms": 0.02, "gpixel_steps_per_s": 600.0},
                              "chain_f64_dilate_conn8_steps1500": {"ms": 1.6, "gpixel_steps_per_s": 950.0},
                              "chain_f64_dilate_conn8_steps100": {"ms": 0.3, "gpixel_steps_per_s": 300.0}},
           "reconstruct_4096": {"u8_opening_31x31": {"ms": 3.0, "steps_applied": 600}},
           "fwd_bwd": {"plain_forward_gpixel_steps_per_s": 430.0}}
    fr = bench.dtype_fractions(sec, 152, 64.0, 64.0, 2070.0)
    u8_peak = 152 * 64 * 2070e6 / 2.5
    assert fr["chain_u8_dilate_conn8_steps1500"]["frac"] == pytest.approx(2000e9 / u8_peak)
    assert fr["window_u8_dilate_s13"]["frac"] == pytest.approx(600e9 / (152 * 64 * 2070e6 / 2.0))
    assert fr["chain_f64_dilate_conn8_steps1500"]["frac"] == pytest.approx(950e9 / (152 * 64 * 2070e6 / 3.0))
    assert "chain_f64_dilate_conn8_steps100" not in fr
    rec = fr["reconstruct_4096_u8_opening_31x31"]
    assert rec["algorithmic_steps"] == 573  # 572 changing steps in the oracle, plus the step that changes nothing
    assert rec["frac"] == pytest.approx(4096 * 4096 * 573 / 3e-3 / u8_peak)
    assert fr["workload4_plain_forward_f32"]["frac"] == pytest.approx(430e9 / (152 * 64 * 2070e6 / 3.0))
