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
    assert lib.bp_backproject_batched(None, None, None, None, 0, None) == 1
    assert "NULL" in lib.bp_last_error().decode()
    lib.bp_destroy(None)  # no-op


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(bp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bp, "_lib", None)
    with pytest.raises(bp.BPError, match="not built"):
        bp.lib()
