"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/psms.h (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "psms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psms_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("psms_create", "psms_dw_apply", "psms_solve", "psms_logdet_ratio", "psms_gauge_sweep",
              "psms_filter_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1204_1306_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1204_1306_gb300 as ps
    with pytest.raises(RuntimeError):
        ps._lib = None
        ps.load_library(str(tmp_path / "nope.so"))
    ps._lib = None


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the compiled library the binding raises."""
    import pytest

    import paper_1204_1306_gb300 as ps
    cached, ps._lib = ps._lib, None
    try:
        with pytest.raises(RuntimeError):
            ps.load_library(str(tmp_path / "libpsms.so"))
    finally:
        ps._lib = cached
