"""C ABI: the library loads, exports every function include/bp.h declares, and rejects bad
arguments on the host before touching a GPU.  CPU only (no compute call)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_1608_03589_gb300 import bp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return bp.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bp_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    want = {"bp_plan_create", "bp_filter", "bp_backproject_direct", "bp_backproject_fourier", "bp_radon",
            "bp_destroy"}
    assert want <= set(_declared())


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(bp.SYMBOLS)


def test_version(lib):
    assert lib.bp_version().decode().startswith("bp ")


def test_plan_create_rejects_bad_geometry(lib):
    th = np.zeros(4)
    p = th.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for args, frag in [((0, 8, 4, p, 0.1), "N out of range"), ((8, 0, 4, p, 0.1), "n_det"),
                       ((8, 8, 0, p, 0.1), "n_theta"), ((8, 8, 4, None, 0.1), "theta is NULL"),
                       ((8, 8, 4, p, -1.0), "det_spacing"), ((8, 8, 4, p, float("nan")), "det_spacing"),
                       ((100000, 8, 4, p, 0.1), "N out of range")]:
        assert not lib.bp_plan_create(*args)
        assert frag in lib.bp_last_error().decode()
    bad = np.array([0.0, np.inf, 1.0, 2.0])
    assert not lib.bp_plan_create(8, 8, 4, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.1)
    assert "non-finite" in lib.bp_last_error().decode()


def test_calls_reject_null_plan(lib):
    assert lib.bp_filter(None, None, 0, None, 0, 0.0, 1, None) == 1
    assert lib.bp_backproject_direct(None, None, 0, None, 1, 0, None) == 1
    assert lib.bp_backproject_fourier(None, None, 0, None, 1, None) == 1
    assert lib.bp_radon(None, None, None, 1, 0, None) == 1
    assert lib.bp_fbp_host(None, None, None, 0, 0.0, 1, None) == 1
    assert lib.bp_fbp_direct(None, None, 0, None, 0, 0.0, 1, None) == 1
    assert lib.bp_fbp_fourier(None, None, 0, None, 0, 0.0, 1, None) == 1
    assert lib.bp_backproject_batched(None, None, None, None, 0, None) == 1
    assert "NULL" in lib.bp_last_error().decode()
    lib.bp_destroy(None)  # no-op


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(bp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bp, "_lib", None)
    with pytest.raises(bp.BPError, match="not built"):
        bp.lib()


def test_shape_calls_reject_null_plan(lib):
    shape = (ctypes.c_int * 2)(16, 1)
    assert lib.bp_autotune(None, 0, 0, 1, None, shape, None) == 1
    assert lib.bp_get_shape(None, 0, 0, 1, shape) == 1
    assert lib.bp_set_shape(None, 0, 0, 1, shape) == 1


def test_tuning_cache_round_trip(lib, tmp_path):
    # "op dtype batch N n_det n_theta W sm_count shape0 shape1"; malformed lines are skipped
    src = tmp_path / "tune.txt"
    good = ["0 0 1 2048 2048 1800 96 152 16 2", "0 1 256 2048 2048 1800 96 152 32 1",
            "1 0 8 1024 1024 720 96 152 4 3"]
    bad = ["0 0 1 2048 2048 1800 96 152 12 2",   # stage 12 invalid
           "1 0 1 64 64 48 96 152 3 1",           # 3 angles per CTA invalid
           "7 0 1 64 64 48 96 152 4 1",           # unknown op
           "0 0 1 2048 2048 1800 96 152 16",      # too short
           "0 0 1 2048 2048 1800 96 152 16 2 9",  # trailing field
           "garbage"]
    src.write_text("\n".join(good[:2] + bad + good[2:]) + "\n")
    bp.tune_cache_load(str(src))
    out = tmp_path / "saved.txt"
    bp.tune_cache_save(str(out))
    saved = set(out.read_text().split("\n")) - {""}
    assert set(good) <= saved
    assert not any(b in saved for b in bad)
    # a radon entry's dtype is normalised to 0
    src2 = tmp_path / "radon.txt"
    src2.write_text("1 2 4 512 512 360 96 152 2 5\n")
    bp.tune_cache_load(str(src2))
    bp.tune_cache_save(str(out))
    assert "1 0 4 512 512 360 96 152 2 5" in out.read_text()


def test_tuning_cache_load_errors(lib, tmp_path):
    with pytest.raises(bp.BPError, match="cannot open"):
        bp.tune_cache_load(str(tmp_path / "absent.txt"))
    junk = tmp_path / "junk.txt"
    junk.write_text("not a tuning line\n")
    with pytest.raises(bp.BPError, match="no valid tuning entry"):
        bp.tune_cache_load(str(junk))
