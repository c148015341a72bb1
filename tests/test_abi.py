"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
and exports every function that include/geomorph.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("#"))
        names += re.findall(r"GEO_API\s+[\w\s\*]*?\b(\w+)\s*\(", src)
    return names


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("geo_dilate_chain", "geo_erode_chain", "geo_reconstruct", "morph_window_dilate",
                     "morph_window_erode", "geo_status_string", "geo_device_status"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1911_13074_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings():
    import paper_1911_13074_gb300 as gm
    lib = gm.load()
    assert lib.geo_status_string(0) == b"GEO_OK"
    for code in range(-7, 0):
        assert lib.geo_status_string(code).startswith(b"GEO_ERR_")


def test_host_argument_checks_need_no_device():
    """Calls rejected on the host return their status before touching the GPU."""
    import paper_1911_13074_gb300 as gm
    lib = gm.load()
    # bad dtype, bad connectivity, pitch < width, negative steps
    assert lib.geo_dilate_chain(7, 16, 16, 16, 4, 4, 4, 8, 3, None) == -2
    assert lib.geo_dilate_chain(0, 16, 16, 16, 4, 4, 4, 6, 3, None) == -1
    assert lib.geo_dilate_chain(0, 16, 16, 16, 4, 4, 3, 8, 3, None) == -1
    assert lib.geo_erode_chain(0, 16, 16, 16, 4, 4, 4, 8, -1, None) == -1
    assert lib.morph_window_dilate(1, 16, 32, 4, 4, 4, -2, None) == -1
    assert lib.geo_reconstruct(0, 16, 16, 16, 4, 4, 4, 8, 3, 0, None, None) == -1
    # empty images are a no-op
    assert lib.geo_dilate_chain(0, None, None, None, 0, 5, 5, 8, 3, None) == 0
    assert lib.morph_window_erode(2, None, None, 3, 0, 0, 4, None) == 0
    # misaligned float pointer, mask overlapping out
    assert lib.geo_dilate_chain(1, 18, 64, 128, 2, 2, 2, 8, 1, None) == -3
    assert lib.geo_dilate_chain(0, 0x1000, 0x2000, 0x2000, 2, 2, 2, 8, 1, None) == -1


def test_probe_rejects_bad_arguments_on_the_host():
    import paper_1911_13074_gb300 as gm
    lib = gm.load()
    r, c = ctypes.c_double(), ctypes.c_double()
    assert lib.geo_probe_minmax_rate(4, ctypes.byref(r), ctypes.byref(c), None) == -1
    assert lib.geo_probe_minmax_rate(-1, ctypes.byref(r), ctypes.byref(c), None) == -1
    assert lib.geo_probe_minmax_rate(0, None, ctypes.byref(c), None) == -1


def test_tune_cache_file_round_trip(tmp_path):
    """The tune-cache text format loads into the table (no device needed)."""
    import paper_1911_13074_gb300 as gm
    path = tmp_path / "tune.txt"
    path.write_text("geomorph-tune 1 Some_GPU\n"
                    "0 0 8 1024 1024 64 20 1.08\n"
                    "1 2 4 300 200 -1 12 0.50\n"
                    "not an entry\n")
    gm.tune_load(path)
    assert gm.tune_lookup(0, 0, 8, 1024, 1024, 1500) == 20   # long chains share the class 64
    assert gm.tune_lookup(0, 0, 8, 1024, 1024, 40) == 0      # a short chain is its own class
    assert gm.tune_lookup(1, "dilate_rec", 4, 300, 200, 0) == 12
    assert gm.tune_lookup(2, 0, 8, 1024, 1024, 1500) == 0
    bad = tmp_path / "bad.txt"
    bad.write_text("something else\n")
    import pytest as _pt
    with _pt.raises(gm.GeoError):
        gm.tune_load(bad)


def test_tune_cache_version_2_round_trip(tmp_path):
    """Version 2: exact entries (E) with a shape variant and the default
    shape's K, size-class entries (C, half-octave classes floor(2 log2 n))
    that other sizes of the class take, and the batch policy (B); a save
    writes the same table back; reset empties it (no device needed)."""
    import paper_1911_13074_gb300 as gm
    gm.tune_reset()
    try:
        path = tmp_path / "tune.txt"
        path.write_text("geomorph-tune 2 Some_GPU\n"
                        "E 0 0 8 300 260 64 12 1 0.40 16 0.45\n"
                        "C 0 0 8 16 16 64 12 1 0.40 16 0.45 1000\n"
                        "C 1 3 4 20 21 -1 8 2 1.00 20 1.20 5000\n"
                        "B 20.0 110.5\n")
        gm.tune_load(path)
        assert gm.tune_lookup(0, 0, 8, 300, 260, 1500) == 16      # the default shape's K
        assert gm.tune_lookup(0, 0, 8, 330, 300, 700) == 16       # same classes: 2 log2 330 = 16.7
        assert gm.tune_lookup(0, 0, 8, 400, 260, 700) == 0        # 2 log2 400 = 17.3: another class
        assert gm.tune_lookup(1, "erode_rec", 4, 1024, 1500, 0) == 20  # classes 20 and 21
        out = tmp_path / "saved.txt"
        gm.tune_save(out)
        lines = out.read_text().splitlines()
        assert lines[0].startswith("geomorph-tune 2 ")
        assert "E 0 0 8 300 260 64 12 1 0.4000 16 0.4500 0" in lines
        assert any(ln.startswith("C 1 3 4 20 21 -1 8 2 ") for ln in lines)
        assert any(ln.startswith("B 20.0000 ") for ln in lines)
        gm.tune_reset()
        assert gm.tune_lookup(0, 0, 8, 300, 260, 1500) == 0
        gm.tune_load(out)
        assert gm.tune_lookup(0, 0, 8, 330, 300, 700) == 16
    finally:
        gm.tune_reset()


def test_missing_library_fails_loudly():
    """No CPU fallback: when the CUDA library cannot be loaded, the first call
    raises instead of computing anything."""
    import subprocess
    import sys
    code = ("import torch, paper_1911_13074_gb300 as m\n"
            "m.dilate_chain(torch.zeros(4, 4, dtype=torch.uint8), torch.zeros(4, 4, dtype=torch.uint8), 3)\n")
    env = dict(os.environ, GEOMORPH_LIB=os.path.join(ROOT, "no_such_dir", "libgeomorph.so"))
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode != 0
    assert "OSError" in p.stderr or "TypeError" in p.stderr
    code2 = "import paper_1911_13074_gb300 as m\nm.load()\n"
    p = subprocess.run([sys.executable, "-c", code2], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode != 0 and "OSError" in p.stderr


def test_cpu_tensors_are_rejected():
    import torch
    import paper_1911_13074_gb300 as m
    a = torch.zeros(4, 4, dtype=torch.uint8)
    with pytest.raises(TypeError):
        m.dilate_chain(a, a, 3)
    with pytest.raises(TypeError):
        m.qdt(a)
