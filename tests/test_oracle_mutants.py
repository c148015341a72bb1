"""Mutation check of the oracle pins: plant plausible mistakes in copies of
oracle.c (on the CPU) and require that the pins catch every one of them."""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle_ops_pins as ops_pins
from tests import test_oracle_pins as pins
from tests import test_oracle_qdt_pins as qdt_pins
from tests import test_oracle_gran_pins as gran_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, original text, mutated text, pins expected to notice)
MUTANTS = [
    ("drop_right_column", "for (int dx = -1; dx <= 1; ++dx) {\n            if (!ora_in_shape",
     "for (int dx = -1; dx <= 0; ++dx) {\n            if (!ora_in_shape"),
    ("clamp_direction", "if (op == ORA_DILATE) v = (mv < v) ? mv : v;",
     "if (op == ORA_DILATE) v = (mv > v) ? mv : v;"),
    ("erode_clamp_direction", "else                  v = (mv > v) ? mv : v;",
     "else                  v = (mv < v) ? mv : v;"),
    ("clip_last_row", "if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;\n            double v",
     "if (qy < 0 || qy >= H - 1 || qx < 0 || qx >= W) continue;\n            double v"),
    ("cross_missing_vertical", "return conn == 8 || dy == 0 || dx == 0;", "return conn == 8 || dy == 0;"),
    ("extra_step", "for (long s = 0; s < steps; ++s) {", "for (long s = 0; s <= steps; ++s) {"),
    ("window_short_right", "x1 = x + s >= W ? W - 1 : x + s;", "x1 = x + s >= W ? W - 1 : x + s - (s > 0);"),
    ("window_rows_short", "y1 = y + s >= H ? H - 1 : y + s;", "y1 = y + s >= H ? H - 1 : y + s - (s > 1);"),
    ("reconstruct_partial_check", "for (long i = 0; i < n; ++i) {\n            if (tmp[i] != out[i])",
     "for (long i = 0; i < n / 2; ++i) {\n            if (tmp[i] != out[i])"),
    ("tie_highest_index", "(op == ORA_DILATE ? (v > best) : (v < best))",
     "(op == ORA_DILATE ? (v >= best) : (v < best))"),
    ("erode_tie_highest_index", "(op == ORA_DILATE ? (v > best) : (v < best))",
     "(op == ORA_DILATE ? (v > best) : (v <= best))"),
    ("mask_wins_ties", "int to_mask = (op == ORA_DILATE) ? (mv < v) : (mv > v);",
     "int to_mask = (op == ORA_DILATE) ? (mv <= v) : (mv > v);"),
    ("gather_transposed", "long py = y - dy, px = x - dx;", "long py = y + dy, px = x + dx;"),
    ("gmask_overwrites", "if (to_mask) gmask[y * W + x] += gmarker[y * W + x];",
     "if (to_mask) gmask[y * W + x] = gmarker[y * W + x];"),
    ("hmax_no_floor", "mk[i] = d < lo ? lo : d;", "mk[i] = d;"),
    ("hmax_adds_h", "double d = ora_sub(f[i], h, f32);", "double d = ora_sub(f[i], -h, f32);"),
    ("hfill_uses_min", "for (long i = 1; i < n; ++i) if (f[i] > mx) mx = f[i];",
     "for (long i = 1; i < n; ++i) if (f[i] < mx) mx = f[i];"),
    ("border_misses_last_column", "(y == 0 || x == 0 || y == H - 1 || x == W - 1)", "(y == 0 || x == 0 || y == H - 1)"),
    ("open_rec_dilates", "if (oracle_window(f, mk, H, W, s, ORA_ERODE) != 0)",
     "if (oracle_window(f, mk, H, W, s, ORA_DILATE) != 0)"),
    ("qdt_ties_take_latest", "if (res > r[i]) { r[i] = res; d[i] = (double)j; }",
     "if (res >= r[i]) { r[i] = res; d[i] = (double)j; }"),
    ("qdt_index_off_by_one", "if (res > r[i]) { r[i] = res; d[i] = (double)j; }",
     "if (res > r[i]) { r[i] = res; d[i] = (double)(j - 1); }"),
    ("qdt_skips_last_erosion", "for (long j = 1; j <= steps; ++j) {", "for (long j = 1; j < steps; ++j) {"),
    ("qdt_residual_dilates", "oracle_step(cur, NULL, nxt, H, W, conn, ORA_ERODE);",
     "oracle_step(cur, NULL, nxt, H, W, conn, ORA_DILATE);"),
    ("eta_drops_plus_one", "tmp[i] = (out[i] - eps[i] > 1.0) ? eps[i] + 1.0 : out[i];",
     "tmp[i] = (out[i] - eps[i] > 1.0) ? eps[i] : out[i];"),
    ("eta_threshold_two", "tmp[i] = (out[i] - eps[i] > 1.0) ? eps[i] + 1.0 : out[i];",
     "tmp[i] = (out[i] - eps[i] > 2.0) ? eps[i] + 1.0 : out[i];"),
    ("opening_dilates_first", "return ora_open_close(f, out, H, W, s, ORA_ERODE);\n}\n\nint oracle_closing",
     "return ora_open_close(f, out, H, W, s, ORA_DILATE);\n}\n\nint oracle_closing"),
    ("open_close_second_step_short", "if (rc == 0) rc = oracle_chain(tmp, NULL, out, H, W, 8, second_op, s);",
     "if (rc == 0) rc = oracle_chain(tmp, NULL, out, H, W, 8, second_op, s > 1 ? s - 1 : s);"),
    ("granulometry_previous_size", "if (ora_open_close(f, g, H, W, s, ORA_ERODE) != 0) { free(g); return -1; }",
     "if (ora_open_close(f, g, H, W, s > 0 ? s - 1 : 0, ORA_ERODE) != 0) { free(g); return -1; }"),
    ("asf_closing_first", "if (ora_open_close(out, tmp, H, W, k, ORA_ERODE) != 0) { free(tmp); return -1; }\n"
     "        if (ora_open_close(tmp, out, H, W, k, ORA_DILATE) != 0)",
     "if (ora_open_close(out, tmp, H, W, k, ORA_DILATE) != 0) { free(tmp); return -1; }\n"
     "        if (ora_open_close(tmp, out, H, W, k, ORA_ERODE) != 0)"),
    ("asf_skips_last_level", "for (long k = 1; k <= s; ++k) {\n        if (ora_open_close(out",
     "for (long k = 1; k < s; ++k) {\n        if (ora_open_close(out"),
]

PIN_TESTS = [
    lambda: pins.test_window_matches_bruteforce_and_chain_on_tiny_images("dilate"),
    lambda: pins.test_window_matches_bruteforce_and_chain_on_tiny_images("erode"),
    lambda: pins.test_four_connected_chain_is_clipped_diamond("dilate"),
    lambda: pins.test_masked_chain_threshold_decomposition(4, "dilate", "u8few"),
    lambda: pins.test_masked_chain_threshold_decomposition(8, "erode", "u8few"),
    lambda: pins.test_reconstruct_is_widest_path(8, "dilate", "u8"),
    lambda: pins.test_reconstruct_is_widest_path(4, "erode", "f64"),
    lambda: pins.test_backward_matches_finite_differences(8, "dilate"),
    lambda: pins.test_backward_source_identity(4, "erode"),
    lambda: pins.test_backward_tie_rule_lowest_index_and_marker_on_mask_tie(),
    lambda: pins.test_backward_erosion_tie_rule(),
    lambda: ops_pins.test_hfill_binary_is_fill_holes(8),
    lambda: ops_pins.test_raobj_binary_removes_border_components(4),
    lambda: ops_pins.test_open_rec_binary_keeps_components_meeting_the_erosion(8),
    lambda: ops_pins.test_hmax_is_widest_path_of_shifted_marker(8, "u8"),
    lambda: ops_pins.test_hmax_flattens_peaks_lower_than_h(),
    lambda: ops_pins.test_hmax_of_image_lower_than_h(),
    lambda: qdt_pins.test_binary_qdt_is_the_distance_transform(8),
    lambda: qdt_pins.test_grey_residuals_match_minimum_filters(4),
    lambda: qdt_pins.test_lipschitz_limit_closed_form(8),
    lambda: gran_pins.test_opening_and_closing_match_scipy(),
    lambda: gran_pins.test_asf_matches_scipy_composition(),
    lambda: gran_pins.test_granulometry_of_separated_squares(),
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, orig, mut, workdir):
    src = open(SRC).read()
    assert orig in src, f"mutation site of {name} not found"
    c_path = os.path.join(workdir, f"{name}.c")
    so_path = os.path.join(workdir, f"{name}.so")
    with open(c_path, "w") as fh:
        fh.write(src.replace(orig, mut, 1))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so_path, c_path])
    prev = oracle.use_library(so_path)
    caught = []
    try:
        for t in PIN_TESTS:
            try:
                t()
            except AssertionError:
                caught.append(t)
                break
    finally:
        oracle.restore_library(prev)
    assert caught, f"no pin detected mutant {name}"
