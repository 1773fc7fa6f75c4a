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


STRUCTS = {
    "LatticeDesc": "psms_lattice_desc", "SolveInfo": "psms_solve_info", "RelGFParams": "psms_relgf_params",
    "FilterParams": "psms_filter_params", "FilterResult": "psms_filter_result", "BlockProblem": "psms_block_problem",
    "TrainParams": "psms_train_params",
}


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    of its C counterpart in include/psms.h (compiled with the host C
    compiler), so no argument is passed at a wrong offset."""
    import shutil
    import subprocess

    import paper_1204_1306_gb300 as ps
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "psms.h"', 'int main(void) {']
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(ps, py)._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for py in STRUCTS:
        cls = getattr(ps, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert got[(py, name)] == getattr(cls, name).offset, (py, name)
